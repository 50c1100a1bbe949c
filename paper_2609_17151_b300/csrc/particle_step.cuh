// particle_step.cuh -- the fused per-species particle step (the hot loop).
//
// One persistent launch per species per step.  Each CTA stages the FP32 node
// field and the species' collision-frequency table into shared memory with a
// bulk asynchronous copy, then streams a contiguous range of particles in
// chunks of two (vector loads and stores; each thread's loads of its next
// chunk are in flight while it computes the current one), doing for each
// particle:
//   gather E^n (linear)  ->  Boris v^{n-1/2} -> v^{n+1/2}  ->  x^{n+1}
//   -> electrode absorption (+ secondary emission)  ->  null-collision MCC
//   -> append of the ionization products  ->  fixed-point CIC deposit of
//   rho^{n+1} into a shared-memory histogram, flushed once per CTA.
// Particle state is updated in place; absorbed particles get cell = -1 and
// are compacted by the next counting sort.
#pragma once
#include "pic_device.cuh"
#include <cooperative_groups.h>

namespace pic {

__device__ __forceinline__ unsigned smem_addr(const void *p)
{
    return (unsigned)__cvta_generic_to_shared(p);
}

// Stage `bytes` (multiple of 16, 16-byte aligned) from global to shared with a
// bulk copy tracked by an mbarrier (issued by one thread).
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, unsigned bytes, uint64_t *mbar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n"
                 :: "r"(smem_addr(dst)), "l"(src), "r"(bytes), "r"(smem_addr(mbar)) : "memory");
}

__device__ __forceinline__ void mbar_init(uint64_t *mbar, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" :: "r"(smem_addr(mbar)), "r"(count) : "memory");
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *mbar, unsigned bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" :: "r"(smem_addr(mbar)), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *mbar, unsigned parity)
{
    unsigned ok;
    asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
                 : "=r"(ok) : "r"(smem_addr(mbar)), "r"(parity) : "memory");
    return ok != 0;
}

// Bounded wait for a staging copy: gives up after `polls` polls and raises
// kErrTimeout.  A copy that was issued may still be in flight then, writing
// into this CTA's shared memory, so the wait goes on (bounded by kDrainPolls,
// whatever `polls` is) until it lands before the caller leaves.  Returns
// false if the data did not arrive within `polls`.
constexpr int kDrainPolls = 1 << 22;
constexpr unsigned kDefaultWaitPolls = 1u << 22;
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *mbar, Ctrl *ctrl, unsigned parity, unsigned polls)
{
    for (unsigned i = 0; i < polls; ++i)
        if (mbar_try_wait(mbar, parity)) return true;
    atomicOr(&ctrl->err, kErrTimeout);
    for (int i = 0; i < kDrainPolls; ++i)
        if (mbar_try_wait(mbar, parity)) return false;
    return false;
}

// Position of eps on the table grid (linear in ln eps), computed once per
// collision candidate and shared by every process's table.
struct GridPos {
    int i;
    float t;
};
__device__ __forceinline__ GridPos grid_pos(float eps, float inv_dlog)
{
    float s = logf(eps * (1.0f / kGridEmin)) * inv_dlog;
    s = fminf(fmaxf(s, 0.0f), (float)(kNGrid - 1));
    const int i = min((int)s, kNGrid - 2);
    return GridPos{i, s - (float)i};
}
// nu_k(eps) between the grid energies; zero below the process threshold
__device__ __forceinline__ float nu_at(const float *tab, GridPos g, float eps, float thr)
{
    if (eps < thr) return 0.0f;
    return (1.0f - g.t) * tab[g.i] + g.t * tab[g.i + 1];
}

// Event counts of one thread over a work item (registers; reduced per warp
// and added to the case's counters once per item).
struct EvCount {
    unsigned cand, coll[kMaxProc], iz, absorbed[2], see, see0, renew;
};
__device__ __forceinline__ void count_proc(EvCount &ev, int proc)
{
#pragma unroll
    for (int k = 0; k < kMaxProc; ++k) ev.coll[k] += (k == proc) ? 1u : 0u;
}

struct Cell { int c; float o; };

// First collision clock of a particle of species sp created (or loaded) in
// `step`: a gap from word 0 of its own block-kBlkGap draw (0 without MCC).
__device__ __forceinline__ uint32_t first_clock(const StepConst &P, int sp, uint32_t id, uint32_t step)
{
    const float lam = P.push.sp[sp].lam;
    if (!(lam > 0.0f)) return 0u;
    return clock_state(u01(draw(P, id, step, sp, kBlkGap).x), lam);
}

// Particles a CTA appends (ionization products, secondary electrons) are
// staged in shared memory, up to kAppendCap per species, and written out at
// the end of its work item after one reservation on each species' counter
// (append_flush): an appending lane then waits on a shared atomic, not on a
// global one that returns.  A case that can append (an ionization process,
// or secondary emission by ions) has the buffer; the others none.
constexpr unsigned kAppendCap = 256;
constexpr int kAppendArrays = 6;                        // cell word, off, vx, vy, vz, id
__host__ __device__ inline unsigned append_cap(const StepConst &P)
{
    if (P.n_species > 1 && !P.periodic && P.see_gamma > 0.0f) return kAppendCap;
    const SpConst &S = P.sp[0];
    if (S.mcc == 1)
        for (int k = 0; k < S.nproc && k < kMaxProc; ++k)
            if (S.kind[k] == PIC_IONIZATION) return kAppendCap;
    return 0u;
}
struct AppBuf {
    uint32_t *base;                                     // [2 species][kAppendArrays][cap] words
    unsigned cap;                                       // entries per species (0: no buffer)
    unsigned *n;                                        // [2] entries taken (may pass cap)
};

// Append one particle to species `sp`, with its first collision clock; deposit
// it into rho^{n+1} directly and add it to the diagnostic-step moments.  The
// lanes of a warp that append together take consecutive entries of the CTA's
// buffer with one shared atomic (the group of lanes active here); once the
// buffer is full they reserve slots of the species' arrays with one global
// atomic and store there.  A slot beyond the capacity raises kErrCapacity and
// the particle is dropped (its deposit is already made: the case is in error).
__device__ void append_particle(const StepConst &P, const AppBuf &ab, int sp, int half, int c, float o, float vx,
                                float vy, float vz, uint32_t id, uint32_t step, bool diag)
{
    Ctrl *ctrl = P.ctrl;
    const uint32_t cw = (uint32_t)c | (first_clock(P, sp, id, step) << kCellBits);
    unsigned k = ab.cap;
    if (ab.cap != 0u) {
        const cooperative_groups::coalesced_group g = cooperative_groups::coalesced_threads();
        unsigned k0 = 0u;
        if (g.thread_rank() == 0) k0 = atomicAdd(&ab.n[sp], g.size());
        k = g.shfl(k0, 0) + g.thread_rank();
    }
    if (k < ab.cap) {
        uint32_t *a = ab.base + (size_t)sp * kAppendArrays * ab.cap + k;
        a[0] = cw;
        a[ab.cap] = __float_as_uint(o);
        a[2 * ab.cap] = __float_as_uint(vx);
        a[3 * ab.cap] = __float_as_uint(vy);
        a[4 * ab.cap] = __float_as_uint(vz);
        a[5 * ab.cap] = id;
    } else {
        const cooperative_groups::coalesced_group g = cooperative_groups::coalesced_threads();
        unsigned long long base = 0ull;
        if (g.thread_rank() == 0) base = atomicAdd(&ctrl->n_total[sp], (unsigned long long)g.size());
        const unsigned long long slot = g.shfl(base, 0) + g.thread_rank();
        if (slot >= P.cap[sp]) {
            atomicOr(&ctrl->err, kErrCapacity);
        } else {
            const SpeciesBufs &B = P.buf[sp][half];
            B.cell[slot] = (int)cw;
            B.off[slot] = o; B.vx[slot] = vx; B.vy[slot] = vy; B.vz[slot] = vz; B.id[slot] = id;
            if (B.z) B.z[slot] = 0.0f;
        }
    }
    const uint32_t f = __float2uint_rz(o * 4294967296.0f);
    unsigned long long *R = P.R[sp] + (size_t)(blockIdx.x % kDepositCopies) * P.r_stride;
    atomicAdd(&R[c], (1ull << 32) - f);
    atomicAdd(&R[c + 1], (unsigned long long)f);
    if (diag) {
        const SpConst &S = P.sp[sp];
        const float v2 = vx * vx + vy * vy + vz * vz;
        const float eps = S.m_over_2e * v2;
        const int nn = P.n_nodes;
        const int c1 = (P.periodic && c + 1 == P.n_cells) ? 0 : c + 1;
        const double iv0 = (!P.periodic && c == 0) ? 1.0 / P.vol_wall : 1.0 / P.vol_interior;
        const double iv1 = (!P.periodic && c1 == P.n_cells) ? 1.0 / P.vol_wall : 1.0 / P.vol_interior;
        atomicAdd(&P.en_sum[sp * nn + c], S.w * (double)eps * (1.0 - (double)o) * iv0);
        atomicAdd(&P.en_sum[sp * nn + c1], S.w * (double)eps * (double)o * iv1);
        atomicAdd(&P.ke_sum[sp], 0.5 * S.m * S.w * (double)v2);
        const float xi = (float)c + o;
        if (sp == 0 && xi >= P.eepf_lo && xi < P.eepf_hi) {
            const int b = (int)(eps * 4.0f);
            if (b < kEepfBins) atomicAdd(&P.eepf[b], 1ull);
        }
    }
}

__device__ __forceinline__ uint4 draw(const CasePush &C, uint32_t id, uint32_t step, int sp, uint32_t blk)
{
    return philox4x32_10(make_uint4(id, step, ((uint32_t)sp << 16) | blk, 0u), C.key0, C.key1);
}

// Electron collision candidate (null-collision method): the process from
// word 1 of the step's block-0 draw r, the direction from words 2-3; v is
// updated for a real collision.  An ionization sets eej, the energy of the
// ejected electron (otherwise left negative): the products are made by
// ionization_products, 32 at a time.
__device__ __forceinline__ void collide_electron(const StepConst &P, const CasePush &C, const float *nus,
                                                 uint32_t id, uint32_t step, float3 &v, EvCount &ev, const uint4 r,
                                                 float &eej_out)
{
    const SpConst &S = P.sp[0];
    ev.cand++;
    const float v2 = v.x * v.x + v.y * v.y + v.z * v.z;
    const float eps = S.m_over_2e * v2;
    const float x = u01(r.y) * S.numax;
    int proc = -1, kind = 0;
    float thr = 0.0f;
    if (S.mcc == 2) {
        proc = 0;
    } else {
        const GridPos g = grid_pos(eps, P.inv_dlog);
        float cum = 0.0f;
        for (int k = 0; k < S.nproc; ++k) {
            cum += nu_at(nus + k * kNGrid, g, eps, S.thr[k]);
            if (x < cum) { proc = k; kind = S.kind[k]; thr = S.thr[k]; break; }
        }
        if (proc < 0) return;
    }
    count_proc(ev, proc);
    const float3 n = iso_dir(u01(r.z), u01(r.w));
    if (kind == 0) {                                    // elastic, atom at rest
        const float speed = sqrtf(v2);
        const float cchi = speed > 0.0f ? (v.x * n.x + v.y * n.y + v.z * n.z) / speed : 1.0f;
        const float epsn = eps * (1.0f - S.recoil * (1.0f - cchi));
        const float sp = S.v_of_sqrt_eps * sqrtf(fmaxf(epsn, 0.0f));
        v = make_float3(sp * n.x, sp * n.y, sp * n.z);
    } else if (kind == 1) {                             // excitation
        const float sp = S.v_of_sqrt_eps * sqrtf(fmaxf(eps - thr, 0.0f));
        v = make_float3(sp * n.x, sp * n.y, sp * n.z);
    } else {                                            // ionization: share eps - thr
        const uint4 a = draw(C, id, step, 0, kBlkAux);
        const float avail = fmaxf(eps - thr, 0.0f);
        const float eej = u01(a.x) * avail;
        const float esc = avail - eej;
        const float sp = S.v_of_sqrt_eps * sqrtf(esc);
        v = make_float3(sp * n.x, sp * n.y, sp * n.z);
        eej_out = eej;
        ev.iz++;
    }
}

// The products of an ionization by electron `id` at (c, o): the ejected
// electron (energy eej, direction from words 1-2 of the block-kBlkAux draw)
// and, with ions, the new ion (Maxwellian at the gas temperature), with the
// ids of the block-kBlkChild draw.
__device__ __forceinline__ void ionization_products(const StepConst &P, const CasePush &C, const AppBuf &ab,
                                                    uint32_t id, uint32_t step, int c, float o, float eej,
                                                    int half_e, int half_i, bool diag)
{
    const SpConst &S = P.sp[0];
    const uint4 a = draw(C, id, step, 0, kBlkAux);
    const uint4 ids = draw(C, id, step, 0, kBlkChild);
    const float3 ne = iso_dir(u01(a.y), u01(a.z));
    const float spe = S.v_of_sqrt_eps * sqrtf(eej);
    append_particle(P, ab, 0, half_e, c, o, spe * ne.x, spe * ne.y, spe * ne.z, ids.x, step, diag);
    if (P.n_species > 1) {
        const uint4 b = draw(C, id, step, 0, kBlkNewIon);
        const float2 g01 = box_muller(u01(b.x), u01(b.y));
        const float2 g23 = box_muller(u01(b.z), u01(b.w));
        const float vt = S.vt_newion;
        append_particle(P, ab, 1, half_i, c, o, vt * g01.x, vt * g01.y, vt * g23.x, ids.y, step, diag);
    }
}

// Ion collision candidate: gas partner from block 1, process from word 1 of
// the block-0 draw r, centre-of-mass direction from its words 2-3.
__device__ __forceinline__ void collide_ion(const StepConst &P, const CasePush &C, const float *nus, uint32_t id,
                                            uint32_t step, float3 &v, EvCount &ev, const uint4 r)
{
    const SpConst &S = P.sp[1];
    ev.cand++;
    const uint4 a = draw(C, id, step, 1, kBlkAux);
    const float2 g01 = box_muller(u01(a.x), u01(a.y));
    const float2 g23 = box_muller(u01(a.z), u01(a.w));
    const float3 vg = make_float3(S.vt_gas * g01.x, S.vt_gas * g01.y, S.vt_gas * g23.x);
    const float3 g = make_float3(v.x - vg.x, v.y - vg.y, v.z - vg.z);
    const float g2 = g.x * g.x + g.y * g.y + g.z * g.z;
    const float eps = S.mu_over_2e * g2;
    const float x = u01(r.y) * S.numax;
    const GridPos gp = grid_pos(eps, P.inv_dlog);
    float cum = 0.0f;
    int proc = -1, kind = 3;
    for (int k = 0; k < S.nproc; ++k) {
        cum += nu_at(nus + k * kNGrid, gp, eps, S.thr[k]);
        if (x < cum) { proc = k; kind = S.kind[k]; break; }
    }
    if (proc < 0) return;
    count_proc(ev, proc);
    if (kind == 4) {                                    // charge exchange
        v = vg;
    } else {                                            // isotropic in the centre-of-mass frame
        const float3 n = iso_dir(u01(r.z), u01(r.w));
        const float f = S.Mfrac * sqrtf(g2);
        v = make_float3(S.mfrac * v.x + S.Mfrac * vg.x + f * n.x, S.mfrac * v.y + S.Mfrac * vg.y + f * n.y,
                        S.mfrac * v.z + S.Mfrac * vg.z + f * n.z);
    }
}

// Secondary electron from an ion that reached electrode `wall`.
__device__ __forceinline__ void emit_secondary(const StepConst &P, const AppBuf &ab, uint32_t id, uint32_t step,
                                               int wall, int half_e, bool diag, EvCount &ev)
{
    const uint4 r = draw(P, id, step, 1, kBlkSee);
    if (u01(r.x) >= P.see_gamma) return;
    const uint4 b = draw(P, id, step, 1, kBlkSeeV);
    const uint4 ids = draw(P, id, step, 1, kBlkChild);
    const float vn = P.see_vth * sqrtf(-2.0f * logf(u01(r.y)));
    const float2 t = box_muller(u01(b.x), u01(b.y));
    const int N = P.n_cells;
    float d = u01(r.z) * vn * P.see_dtdx;
    if (d >= (float)N) d = 0.5f * (float)N;
    const float fl = floorf(d);
    int c;
    float o;
    if (wall == 0) {
        c = (int)fl; o = d - fl;
    } else {
        c = N - 1 - (int)fl; o = 1.0f - (d - fl);
        if (o >= 1.0f) { o = 0.0f; c += 1; }
        if (c >= N) { c = N - 1; o = 0.99999994f; }
    }
    if (o >= 1.0f) { o = 0.0f; c += 1; }
    if (c >= N) { c = N - 1; o = 0.99999994f; }
    const float vx = wall == 0 ? vn : -vn;
    append_particle(P, ab, 0, half_e, c, o, vx, P.see_vth * t.x, P.see_vth * t.y, ids.x, step, diag);
    ev.see++;
    if (wall == 0) ev.see0++;
}

// Shared deposit histogram, per cell: particle count n and the sum of the
// fixed-point offsets F = sum f split as (F >> 16, F & 0xFFFF), so that every
// counter is a native 32-bit shared atomic (a 64-bit shared add measured
// several times slower where the lanes of a warp share a cell, as sorted
// particles do).  At the flush, node c gets n 2^32 - F and node c+1 gets F
// (exact).  A counter pair holds 65536 particles of one cell (the sums of
// f >> 16 and f & 0xFFFF stay below 2^32); the histogram is flushed when a
// cell passes kCellFlush of them (the count's atomic reports it).  The CTA
// checks the flag (one barrier) every kCellHeadroom / (particles per tile)
// tiles, during which a cell gains at most kCellHeadroom more, so no cell
// exceeds 65536.  Particles spread over many cells (unsorted) are thus
// flushed once per work item.
struct DepHist {
    unsigned *cnt, *fhi, *flo;
    unsigned *full;                                     // set when a cell passed kCellFlush
};
constexpr unsigned kCellFlush = 32768;
constexpr unsigned kCellHeadroom = 32768;

__device__ __forceinline__ void hist_run(const DepHist &h, int c, unsigned n, unsigned long long sf)
{
    if (atomicAdd(&h.cnt[c], n) + n > kCellFlush) *h.full = 1u;
    atomicAdd(&h.fhi[c], (unsigned)(sf >> 16));
    atomicAdd(&h.flo[c], (unsigned)(sf & 0xFFFFull));
}

// Add the CTA's histogram to the global deposit and clear it.
__device__ __forceinline__ void hist_flush(const DepHist &h, int N, unsigned long long *R)
{
    __syncthreads();                                   // every hist_run of the CTA done
    if (threadIdx.x == 0) *h.full = 0u;
    for (int c = threadIdx.x; c < N; c += blockDim.x) {
        const unsigned n = h.cnt[c];
        if (n) {
            const unsigned long long F = ((unsigned long long)h.fhi[c] << 16) + h.flo[c];
            atomicAdd(&R[c], ((unsigned long long)n << 32) - F);
            atomicAdd(&R[c + 1], F);
            h.cnt[c] = 0u; h.fhi[c] = 0u; h.flo[c] = 0u;
        }
    }
    __syncthreads();
}

// Deferred draws: entries of a warp's draw queue (slot index within the work
// item, candidate flag in bit 31).  A chunk of CH particles per lane adds at
// most 32 CH entries, and the queue runs whenever 32 have gathered, so it
// never holds more than 32 CH + 31.  0 without collisions.
__host__ __device__ constexpr int draw_queue_cap(int mcc, int ch) { return mcc != 0 ? 32 * ch + 32 : 0; }
// Ionizations whose products are still to be made, per warp: entries of
// (cell, offset, parent id, eej).  A queue run of 32 draws adds at most 32, and
// products are made whenever 32 have gathered, so 63 at most are waiting.
// Electrons with cross-section tables only.
constexpr int kChildWords = 4;
__host__ __device__ constexpr int child_queue_cap(int sp, int mcc) { return (sp == 0 && mcc == 1) ? 64 : 0; }

// Shared memory layout of the step kernel (bytes, 16-aligned pieces): node
// field, deposit histogram, collision table, diagnostic moments, each warp's
// draw queue (`qcap` 4-byte entries), the append buffer (`apcap` entries a
// species), each warp's queue of ionizations (`ccap` entries).  With `stages` > 0 the particle tiles
// (one 4-particle chunk per thread, `narr` arrays of 16 bytes per chunk) pass
// through `stages` buffers at the end.
__host__ __device__ inline unsigned align16(unsigned x) { return (x + 15u) & ~15u; }
__host__ __device__ inline unsigned align128(unsigned x) { return (x + 127u) & ~127u; }
struct StepSmem {
    unsigned e_off, h_off, nu_off, en_off, eepf_off, q_off, app_off, cq_off, st_off, st_bytes, total;
    __host__ __device__ StepSmem(int n_cells, int nproc, int threads = 0, int stages = 0, int narr = 0,
                                 int qcap = 0, unsigned apcap = 0, int ccap = 0)
    {
        e_off = 0;
        h_off = align16(e_off + (unsigned)n_cells * 8u);
        nu_off = align16(h_off + (unsigned)n_cells * 12u);
        en_off = align16(nu_off + (unsigned)nproc * kNGrid * 4u);
        eepf_off = align16(en_off + (unsigned)(n_cells + 1) * 4u);
        q_off = align16(eepf_off + kEepfBins * 4u);
        app_off = align16(q_off + (unsigned)(threads / 32) * (unsigned)qcap * 4u);
        cq_off = align16(app_off + 2u * kAppendArrays * apcap * 4u);
        const unsigned cq_end = cq_off + (unsigned)(threads / 32) * (unsigned)ccap * kChildWords * 4u;
        st_off = align128(cq_end);
        st_bytes = (unsigned)threads * 16u * (unsigned)narr;      // one stage
        total = stages > 0 ? st_off + (unsigned)stages * st_bytes : align16(cq_end);
    }
};

// Particle arrays a step streams: cell (with the collision clock), off, vx,
// vy, vz.  The id is read only for the particles that draw random numbers in
// the step (the end of a collision clock, secondary emission, axial
// renewal), one load each, from the draw queue or in place.
__host__ __device__ constexpr int step_arrays(int, bool, int) { return 5; }

// Direct-load path: particles per chunk, and how many chunks ahead of the one
// being computed each thread keeps its loads in flight (register double
// buffering; 0 = none).  Within 64 registers a thread, chunks of two with one
// chunk ahead measured fastest on the E x B box: chunks of one with two to
// four ahead, chunks of two with two ahead, and chunks of four without any
// were slower.  The staged path always moves chunks of four.
// Particles a load-time deposit CTA adds to its shared histogram between
// flushes: a cell's sums of f >> 16 and f & 0xFFFF then stay below 2^31.
constexpr int kDepositSpan = 32768;
constexpr int kDirectChunk = 2;
constexpr int kDirectDepth = 1;

// One chunk of CH consecutive particles of a species, in registers.
template <int CH> struct VecOf;
template <> struct VecOf<4> { typedef int4 I; typedef float4 F; typedef uint4 U; };
template <> struct VecOf<2> { typedef int2 I; typedef float2 F; typedef uint2 U; };
template <> struct VecOf<1> { typedef int I; typedef float F; typedef uint32_t U; };
template <int CH> struct Chunk {
    int c[CH];
    float o[CH], vx[CH], vy[CH], vz[CH], z[CH];
};
// vector load / store of CH elements (address aligned to CH elements)
template <class V, int CH, class T>
__device__ __forceinline__ void vload(T (&d)[CH], const T *src)
{
    const V v = *reinterpret_cast<const V *>(src);
    const T *e = reinterpret_cast<const T *>(&v);
#pragma unroll
    for (int q = 0; q < CH; ++q) d[q] = e[q];
}
template <class V, int CH, class T>
__device__ __forceinline__ void vstore(T *dst, const T (&s)[CH])
{
    V v;
    T *e = reinterpret_cast<T *>(&v);
#pragma unroll
    for (int q = 0; q < CH; ++q) e[q] = s[q];
    *reinterpret_cast<V *>(dst) = v;
}
// Chunk starting at element e0 of the arrays of B (cell, off, vx, vy, vz, and
// id, z when asked).
template <int CH, bool Z>
__device__ __forceinline__ void load_chunk(Chunk<CH> &t, const SpeciesBufs &B, unsigned e0)
{
    typedef VecOf<CH> V;
    vload<typename V::I>(t.c, B.cell + e0);
    vload<typename V::F>(t.o, B.off + e0);
    vload<typename V::F>(t.vx, B.vx + e0);
    vload<typename V::F>(t.vy, B.vy + e0);
    vload<typename V::F>(t.vz, B.vz + e0);
    if (Z) vload<typename V::F>(t.z, B.z + e0);
}

// Per-CTA shared state of the particle step besides the dynamic tables.
struct StepShared {
    uint64_t mbar;                                      // staging barrier (phase toggles per item)
    uint64_t full[kMaxStages];                          // particle-tile barriers (phase toggles per use)
    unsigned tile_rel[kMaxStages];                      // warps done reading each buffer (running count)
    unsigned tile_abort;                                // a tile wait gave up: stop streaming
    unsigned s_cnt[2 + 2 * kMaxProc];                   // candidates, per process, ionizations
    unsigned s_abs[2], s_see, s_see0, s_renew;
    unsigned hist_full;                                 // a deposit counter passed kCellFlush
    unsigned app_n[2];                                  // append buffer entries taken, per species
    unsigned long long app_base[2];                     // slots reserved for them at the item's end
    float s_red[2][kStepThreads / 32];
};

// End of a work item: the CTA's staged appends go to the species' arrays, at
// slots reserved with one atomic per species, in coalesced stores.
__device__ __forceinline__ void append_flush(const StepConst &P, const AppBuf &ab, StepShared &sh, int half_e,
                                             int half_i)
{
    __syncthreads();                                    // every append of the CTA staged
    for (int sp = 0; sp < P.n_species; ++sp) {
        const unsigned na = min(ab.n[sp], ab.cap);      // the same for every thread
        if (na == 0u) continue;
        if (threadIdx.x == 0) sh.app_base[sp] = atomicAdd(&P.ctrl->n_total[sp], (unsigned long long)na);
        __syncthreads();
        const unsigned long long base = sh.app_base[sp];
        const SpeciesBufs &B = P.buf[sp][sp == 0 ? half_e : half_i];
        const uint32_t *a = ab.base + (size_t)sp * kAppendArrays * ab.cap;
        for (unsigned i = threadIdx.x; i < na; i += blockDim.x) {
            const unsigned long long slot = base + i;
            if (slot >= P.cap[sp]) {
                atomicOr(&P.ctrl->err, kErrCapacity);
                break;
            }
            B.cell[slot] = (int)a[i];
            B.off[slot] = __uint_as_float(a[ab.cap + i]);
            B.vx[slot] = __uint_as_float(a[2 * ab.cap + i]);
            B.vy[slot] = __uint_as_float(a[3 * ab.cap + i]);
            B.vz[slot] = __uint_as_float(a[4 * ab.cap + i]);
            B.id[slot] = a[5 * ab.cap + i];
            if (B.z) B.z[slot] = 0.0f;
        }
    }
}

// One work item: chunks (CH particles) [beg, end) of the k-th of nk equal
// slices of species SP of one case.  Stages the case's node field and the
// species' table, processes the slice, flushes the deposit, the moments and
// the counters.  `parity` is the staging barrier's phase, toggled per item;
// bit s of `tile_phase` is the phase of tile buffer s.
//
// The slice is processed in tiles of one chunk per thread.  Without STAGED
// each thread loads its chunks (DCHUNK particles each) from global memory
// itself, issuing the loads of chunk k + DDEPTH before it computes chunk k
// (DDEPTH = 0: no look-ahead); with STAGED and
// S.stages = n > 0, n tiles stay in flight as bulk copies (global ->
// shared, completion on a per-buffer mbarrier), so that HBM streams while
// the warps compute, and the warps read their chunk from shared memory.
// Results are written straight back to global memory.
template <int SP, bool PERIODIC, int MCC, bool STAGED, bool AXIAL, int DCHUNK = kDirectChunk,
          int DDEPTH = kDirectDepth>
__device__ __forceinline__ void particle_item(const StepConst &P, const CasePush &C, unsigned char *smem, StepShared &sh,
                                              unsigned &parity, unsigned &tile_phase, long long k_item,
                                              long long n_items)
{
    const SpConst &S = P.sp[SP];
    const SpPush &H = C.sp[SP];                         // push constants (kernel parameter)
    const int N = P.n_cells;
    constexpr int kArr = step_arrays(SP, PERIODIC, MCC);
    const int n_stages = STAGED ? S.stages : 0;
    constexpr int QCAP = draw_queue_cap(MCC, STAGED ? 4 : DCHUNK);
    const unsigned apcap = append_cap(P);
    constexpr int KCAP = child_queue_cap(SP, MCC);
    const StepSmem L(N, MCC == 1 ? S.nproc : 0, blockDim.x, n_stages, kArr, QCAP, apcap, KCAP);
    const AppBuf ab{reinterpret_cast<uint32_t *>(smem + L.app_off), apcap, sh.app_n};
    const float2 *Es = reinterpret_cast<const float2 *>(smem + L.e_off);
    const DepHist hist{reinterpret_cast<unsigned *>(smem + L.h_off), reinterpret_cast<unsigned *>(smem + L.h_off) + N,
                       reinterpret_cast<unsigned *>(smem + L.h_off) + 2 * N, &sh.hist_full};
    float *nus = reinterpret_cast<float *>(smem + L.nu_off);
    float *hen = reinterpret_cast<float *>(smem + L.en_off);
    unsigned *heepf = reinterpret_cast<unsigned *>(smem + L.eepf_off);
    unsigned *s_cnt = sh.s_cnt, *s_abs = sh.s_abs;

    Ctrl *ctrl = P.ctrl;
    const int tid = threadIdx.x;
    const long long n = (long long)ctrl->n_active[SP];
    constexpr int CH = STAGED ? 4 : DCHUNK;              // particles per chunk
    constexpr bool PIPE = !STAGED && DDEPTH > 0;
    const long long n_chunks = (n + CH - 1) / CH;
    long long per = (n_chunks + n_items - 1) / n_items;
    per = (per + 31) & ~31ll;
    const long long beg = k_item * per;
    const long long end = min(beg + per, n_chunks);
    if (beg >= end) return;                             // uniform over the CTA

    const unsigned e_bytes = align16((unsigned)N * 8u);
    const unsigned nu_bytes = MCC == 1 ? (unsigned)S.nproc * kNGrid * 4u : 0u;
    if (tid == 0) {
        asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");   // earlier reads before the async writes
        mbar_expect_tx(&sh.mbar, e_bytes + nu_bytes);
        bulk_g2s(smem + L.e_off, P.E32p, e_bytes, &sh.mbar);
        if (MCC == 1) bulk_g2s(nus, P.nu_tab[SP], nu_bytes, &sh.mbar);
    }
    const long long step_ll = ctrl->step;
    const uint32_t step = (uint32_t)step_ll;
    const bool diag = P.diag_interval > 0 && ((step_ll + 1) % P.diag_interval) == 0;
    for (int j = tid; j < N; j += blockDim.x) { hist.cnt[j] = 0u; hist.fhi[j] = 0u; hist.flo[j] = 0u; }
    if (diag) for (int j = tid; j <= N; j += blockDim.x) hen[j] = 0.0f;
    if (diag) for (int j = tid; j < kEepfBins; j += blockDim.x) heepf[j] = 0u;
    if (tid < 2 + 2 * kMaxProc) s_cnt[tid] = 0u;
    if (tid < 2) s_abs[tid] = 0u;
    if (tid == 0) {
        sh.s_see = 0u; sh.s_see0 = 0u; sh.s_renew = 0u; sh.hist_full = 0u;
        sh.app_n[0] = 0u; sh.app_n[1] = 0u;
    }
    const int half = ctrl->cur[SP];
    const int half_e = ctrl->cur[0];
    const int half_i = P.n_species > 1 ? ctrl->cur[1] : 0;
    const SpeciesBufs B = P.buf[SP][half];
    // The item's particles are addressed from base pointers shifted to its
    // first particle (the same for every thread) with 32-bit offsets.
    const long long item0 = beg * CH;
    SpeciesBufs Bi = B;
    Bi.cell += item0; Bi.off += item0; Bi.vx += item0; Bi.vy += item0; Bi.vz += item0; Bi.id += item0;
    if (AXIAL) Bi.z += item0;
    const unsigned n_ch = (unsigned)(end - beg);                               // chunks of the item
    const unsigned item_n = (unsigned)min(n - item0, (long long)n_ch * CH);   // its particles below n
    const int T = blockDim.x;                           // chunks per tile
    // PIPE: the next D chunks, loads in flight; the first ones are issued
    // before the wait for the node field, so that both arrive together
    constexpr int D = PIPE ? DDEPTH : 1;
    Chunk<CH> nx[D] = {};
    if (PIPE) {
#pragma unroll
        for (int d = 0; d < D; ++d)
            if ((unsigned)(d * T + tid) < n_ch) load_chunk<CH, AXIAL>(nx[d], Bi, (unsigned)(d * T + tid) * CH);
    }

    const bool staged = mbar_wait_bounded(&sh.mbar, ctrl, parity, P.wait_polls);
    parity ^= 1u;
    if (!__syncthreads_and(staged)) return;
    if (n_stages > 0 && sh.tile_abort) return;          // this CTA gave up on its tiles earlier

    const float dtdx = P.dtdx;
    const int lane = tid & 31, warp = tid >> 5;
    float ke_acc = 0.0f, pw_acc = 0.0f;
    EvCount ev{};

    unsigned long long *const R_cta = P.R[SP] + (size_t)(blockIdx.x % kDepositCopies) * P.r_stride;
    const int n_warps = T >> 5;
    const int n_tiles = (int)((end - beg + T - 1) / T);
    unsigned char *const tiles = smem + L.st_off;
    // tile k -> buffer b = k mod n_stages: one bulk copy per array, one mbarrier per buffer
    auto issue_tile = [&](int k, int b) {
        const long long c0 = beg + (long long)k * T;
        const unsigned bytes = (unsigned)min((long long)T, end - c0) * 16u;
        const void *src[6] = {B.cell, B.off, B.vx, B.vy, B.vz, B.id};
        asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");   // earlier reads of the buffer first
        mbar_expect_tx(&sh.full[b], bytes * kArr);
#pragma unroll
        for (int a = 0; a < kArr; ++a)
            bulk_g2s(tiles + ((size_t)(b * kArr + a) * T) * 16u, reinterpret_cast<const char *>(src[a]) + c0 * 16,
                     bytes, &sh.full[b]);
    };
    if (n_stages > 0 && tid == 0)
        for (int k = 0; k < n_tiles && k < n_stages; ++k) issue_tile(k, k);

    // Diagnostic moments of a particle at (c, on) with velocity v^{n+1/2}.
    auto moments = [&](int c, float on, const float3 &v) {
        const float v2 = v.x * v.x + v.y * v.y + v.z * v.z;
        const float eps = S.m_over_2e * v2;
        ke_acc += v2;
        atomicAdd(&hen[c], eps * (1.0f - on));
        atomicAdd(&hen[c + 1], eps * on);
        if (SP == 0) {
            const float xi = (float)c + on;
            if (xi >= P.eepf_lo && xi < P.eepf_hi) {
                const int bin = (int)(eps * 4.0f);
                if (bin < kEepfBins) atomicAdd(&heepf[bin], 1u);
            }
        }
    };
    // Deferred draws.  A particle whose collision clock ends this step needs
    // its random block, a new clock and, if it is a candidate, the collision;
    // a few percent of the particles do each step, scattered over the lanes.
    // Run in place, a warp would pass through that code once per chunk slot
    // whenever any lane needed it, with one or two lanes active.  Instead the
    // chunk is stored with the pushed state, the particle's slot is queued in
    // the warp's part of shared memory, and the queue runs 32 at a time, one
    // per lane, reading the particle back and writing its new clock and
    // velocity over the stored ones.  The results are the same: the draw is
    // keyed by the particle and the step, not by the lane that makes it.
    uint32_t *const Q = reinterpret_cast<uint32_t *>(smem + L.q_off) + warp * QCAP;
    int qn = 0;                                         // entries queued (warp-uniform)
    // Ionizations: the scattered electron is finished in the queue run, the
    // products (two more draws for the ejected electron and the ion, and each
    // one's first collision clock: four Philox blocks) wait in a second
    // per-warp queue and are made 32 at a time, so that the few lanes of a
    // run that ionize do not hold the warp through that code alone.
    uint32_t *const KQ = reinterpret_cast<uint32_t *>(smem + L.cq_off) + warp * KCAP * kChildWords;
    int kn = 0;                                         // ionizations queued (warp-uniform)
    const unsigned lt_mask = (1u << lane) - 1u;
    auto run_children = [&](int j, bool valid) {        // entry j of the ionization queue
        if (SP == 0 && valid)
            ionization_products(P, C, ab, KQ[2 * KCAP + j], step, (int)KQ[j], __uint_as_float(KQ[KCAP + j]),
                                __uint_as_float(KQ[3 * KCAP + j]), half_e, half_i, diag);
    };
    auto run_queue = [&](int j, bool valid) {           // entry j of this warp's draw queue (every lane)
        float eej = -1.0f;
        int c = 0;
        float on = 0.0f;
        uint32_t pid = 0u;
        if (valid) {
            const uint32_t w = Q[j];
            const uint32_t e = w & 0x7fffffffu;
            pid = Bi.id[e];
            c = Bi.cell[e] & kCellMask;
            float3 v = make_float3(Bi.vx[e], Bi.vy[e], Bi.vz[e]);
            on = (diag || (SP == 0 && MCC == 1)) ? Bi.off[e] : 0.0f;   // ionization products, moments
            const uint4 r = draw(C, pid, step, SP, kBlkMcc);
            const uint32_t clk = clock_state(u01(r.x), H.lam);
            if (w >> 31) {
                if (SP == 0) collide_electron(P, C, nus, pid, step, v, ev, r, eej);
                else collide_ion(P, C, nus, pid, step, v, ev, r);
            }
            Bi.cell[e] = c | (int)(clk << kCellBits);
            Bi.vx[e] = v.x; Bi.vy[e] = v.y; Bi.vz[e] = v.z;
            if (diag) moments(c, on, v);
        }
        if (KCAP > 0) {
            const unsigned m = __ballot_sync(0xffffffffu, eej >= 0.0f);
            if (m != 0u) {                              // warp-uniform
                if (eej >= 0.0f) {
                    const int k = kn + __popc(m & lt_mask);
                    KQ[k] = (uint32_t)c;
                    KQ[KCAP + k] = __float_as_uint(on);
                    KQ[2 * KCAP + k] = pid;
                    KQ[3 * KCAP + k] = __float_as_uint(eej);
                }
                kn += __popc(m);
                if (kn >= 32) {
                    kn -= 32;
                    __syncwarp();                       // the entries first
                    run_children(kn + lane, true);
                    __syncwarp();                       // the run's reads before new entries
                }
            }
        }
    };
    const int check_every = max(1, (int)(kCellHeadroom / ((unsigned)T * (unsigned)CH)));
    int check_left = check_every, b = 0;
    for (int k = 0; k < n_tiles; ++k) {
        if (check_left == 0) {                           // uniform over the CTA
            check_left = check_every;
            if (__syncthreads_or(sh.hist_full != 0u)) hist_flush(hist, N, R_cta);
        }
        --check_left;
        const unsigned ci = (unsigned)(k * T + tid);                          // chunk within the item
        bool live_chunk = ci < n_ch;
        if (n_stages > 0) {
            // skip the wait once any warp of the CTA has given up on a tile
            const bool ok = !sh.tile_abort && mbar_wait_bounded(&sh.full[b], ctrl, (tile_phase >> b) & 1u, P.wait_polls);
            tile_phase ^= 1u << b;
            if (!ok) sh.tile_abort = 1u;
            live_chunk = live_chunk && ok;
        }
        const unsigned e0 = ci * CH;                                          // its first particle
        Chunk<CH> t;
        if (PIPE) {
            t = nx[0];
#pragma unroll
            for (int d = 0; d + 1 < D; ++d) nx[d] = nx[d + 1];
            if (ci + (unsigned)(D * T) < n_ch) load_chunk<CH, AXIAL>(nx[D - 1], Bi, e0 + (unsigned)(D * T * CH));
        } else if (live_chunk) {
            if (n_stages > 0) {
                const unsigned char *tl = tiles + ((size_t)b * kArr * T + tid) * 16u;
                const size_t stride = (size_t)T * 16u;
                vload<int4>(t.c, reinterpret_cast<const int *>(tl));
                vload<float4>(t.o, reinterpret_cast<const float *>(tl + stride));
                vload<float4>(t.vx, reinterpret_cast<const float *>(tl + 2 * stride));
                vload<float4>(t.vy, reinterpret_cast<const float *>(tl + 3 * stride));
                vload<float4>(t.vz, reinterpret_cast<const float *>(tl + 4 * stride));
            } else {
                load_chunk<CH, AXIAL>(t, Bi, e0);
            }
        }
        if (n_stages > 0) {
            // Release buffer b: the last warp of the CTA to have read its
            // chunk of tile k refills it with tile k + n_stages (per-buffer
            // arrival counter; block fences order every warp's reads before
            // the bulk copy, which fence.proxy.async hands to the async proxy).
            __syncwarp();
            if (lane == 0) {
                __threadfence_block();
                const unsigned arrived = atomicAdd(&sh.tile_rel[b], 1u) + 1u;
                if (arrived % (unsigned)n_warps == 0u && !sh.tile_abort) {
                    __threadfence_block();
                    if (k + n_stages < n_tiles) issue_tile(k + n_stages, b);
                }
            }
            b = (b + 1 == n_stages) ? 0 : b + 1;
        }
        int (&cc)[CH] = t.c;
        float (&oo)[CH] = t.o;
        float (&vx)[CH] = t.vx;
        float (&vy)[CH] = t.vy;
        float (&vz)[CH] = t.vz;
        float (&za)[CH] = t.z;
        int dc[CH];
        uint32_t df[CH];
        unsigned needm = 0u, candm = 0u;                // bit q: clock ended (queue the draw), candidate
        const int n_valid = live_chunk ? (int)min((unsigned)CH, item_n - e0) : 0;   // particles of the chunk below n
#pragma unroll
        for (int q = 0; q < CH; ++q) {
            dc[q] = -1;
            df[q] = 0;
            int c = cc[q];
            if (q >= n_valid || c < 0) continue;
            uint32_t clk = (uint32_t)c >> kCellBits;     // collision clock 2 k + c
            c &= kCellMask;
            auto pid_of = [&]() -> uint32_t { return Bi.id[e0 + q]; };    // read only when it draws
            float o = oo[q];
            // 1. gather E^n (linear weights), plus the imposed field.  The
            // library is built without implicit multiply-add contraction and
            // every FMA of the push is written out, so that each kernel
            // variant (direct, staged, batched) rounds identically.
            const float2 ep = Es[c];                        // (E_c, E_{c+1})
            const float e_mesh = fmaf(o, ep.y, (1.0f - o) * ep.x);
            const float ex = e_mesh + C.ex_ext;
            // 2. Boris: half kick, rotation, half kick
            const float hx = H.c_e * ex;
            float3 vm = make_float3(vx[q] + hx, vy[q] + H.cEy, vz[q] + H.cEz);
            float3 v;
            if (H.rot == 0) {                               // no magnetic field: two half kicks
                v = make_float3(vm.x + hx, vm.y + H.cEy, vm.z + H.cEz);
            } else if (H.rot == 1) {                        // B along y: rotation in the x-z plane
                const float vpx = fmaf(-vm.z, H.tB[1], vm.x), vpz = fmaf(vm.x, H.tB[1], vm.z);
                v = make_float3(fmaf(-vpz, H.sB[1], vm.x) + hx, vm.y + H.cEy, fmaf(vpx, H.sB[1], vm.z) + H.cEz);
            } else {                                        // v- + v- x t, then v- + v' x s
                const float3 vp = make_float3(vm.x + fmaf(vm.y, H.tB[2], -(vm.z * H.tB[1])),
                                              vm.y + fmaf(vm.z, H.tB[0], -(vm.x * H.tB[2])),
                                              vm.z + fmaf(vm.x, H.tB[1], -(vm.y * H.tB[0])));
                v = make_float3(vm.x + fmaf(vp.y, H.sB[2], -(vp.z * H.sB[1])) + hx,
                                vm.y + fmaf(vp.z, H.sB[0], -(vp.x * H.sB[2])) + H.cEy,
                                vm.z + fmaf(vp.x, H.sB[1], -(vp.y * H.sB[0])) + H.cEz);
            }
            if (diag) pw_acc += v.x * e_mesh;
            // 3. move
            float on = fmaf(v.x, dtdx, o);
            const float fl = floorf(on);
            on -= fl;
            c += (int)fl;
            if (on >= 1.0f) { on = 0.0f; c += 1; }
            if (PERIODIC) {
                if ((unsigned)c >= (unsigned)N) { c %= N; if (c < 0) c += N; }
            } else if ((unsigned)c >= (unsigned)N) {
                // 4. electrode absorption (+ secondary emission by ions)
                const int wall = c < 0 ? 0 : 1;
                ev.absorbed[wall]++;
                if (SP == 1 && P.ifedf_scale > 0.0f) {        // ion energy at the electrode
                    const int bin = (int)(S.m_over_2e * (v.x * v.x + v.y * v.y + v.z * v.z) * P.ifedf_scale);
                    if (bin >= 0 && bin < kIfedfBins) atomicAdd(&P.ifedf[wall * kIfedfBins + bin], 1ull);
                }
                if (SP == 1 && P.see_gamma > 0.0f) emit_secondary(P, ab, pid_of(), step, wall, half_e, diag, ev);
                cc[q] = -1;
                oo[q] = on; vx[q] = v.x; vy[q] = v.y; vz[q] = v.z;
                continue;
            }
            // axial renewal: z advances by v_z dt; at |z| >= L the particle
            // takes a new velocity from the renewal Maxwellian and z = 0
            if (AXIAL) {
                float zn = fmaf(v.z, P.dt_f, za[q]);
                if (fabsf(zn) >= P.axial_len) {
                    const uint4 r = draw(P, pid_of(), step, SP, kBlkRenew);
                    const float2 g01 = box_muller(u01(r.x), u01(r.y));
                    const float2 g23 = box_muller(u01(r.z), u01(r.w));
                    v = make_float3(fmaf(S.renew_vt, g01.x, S.renew_drift[0]), fmaf(S.renew_vt, g01.y, S.renew_drift[1]),
                                    fmaf(S.renew_vt, g23.x, S.renew_drift[2]));
                    zn = 0.0f;
                    ev.renew++;
                }
                za[q] = zn;
            }
            // 5-6. null-collision MCC with v^{n+1/2} at x^{n+1}: the clock counts
            // down; at its end the particle draws (block 0) a fresh gap and, unless
            // the gap was a cut long one, is a collision candidate; products
            // appended.  The draw is queued (see run_queue).
            if (MCC != 0 && H.lam > 0.0f) {
                if (clk >= 2u) {
                    clk -= 2u;
                } else {
                    needm |= 1u << q;
                    candm |= ((clk & 1u) ^ 1u) << q;
                }
            }
            cc[q] = c | (int)(clk << kCellBits); oo[q] = on; vx[q] = v.x; vy[q] = v.y; vz[q] = v.z;
            dc[q] = c;
            df[q] = __float2uint_rz(on * 4294967296.0f);
            if (diag && !((needm >> q) & 1u)) moments(c, on, v);
        }
        // write back (never past n: slots beyond belong to this step's appends)
        if (live_chunk) {
            if (n_valid == CH) {
                typedef VecOf<CH> V;
                vstore<typename V::I>(Bi.cell + e0, cc);
                vstore<typename V::F>(Bi.off + e0, oo);
                vstore<typename V::F>(Bi.vx + e0, vx);
                vstore<typename V::F>(Bi.vy + e0, vy);
                vstore<typename V::F>(Bi.vz + e0, vz);
                if (AXIAL) vstore<typename V::F>(Bi.z + e0, za);
            } else {
#pragma unroll
                for (int q = 0; q < CH; ++q) {
                    if (q >= n_valid) break;
                    Bi.cell[e0 + q] = cc[q]; Bi.off[e0 + q] = oo[q];
                    Bi.vx[e0 + q] = vx[q]; Bi.vy[e0 + q] = vy[q]; Bi.vz[e0 + q] = vz[q];
                    if (AXIAL) Bi.z[e0 + q] = za[q];
                }
            }
        }
        // 7. deposit: merge equal-cell runs in the thread, then one warp-wide
        // reduction when the whole warp's 128 particles share one cell.
        int acc_c = -1;
        unsigned acc_n = 0;
        unsigned long long acc_f = 0;
        bool split = false;
#pragma unroll
        for (int q = 0; q < CH; ++q) {
            if (dc[q] < 0) continue;
            if (dc[q] == acc_c) { acc_n++; acc_f += df[q]; }
            else {
                if (acc_c >= 0) { hist_run(hist, acc_c, acc_n, acc_f); split = true; }
                acc_c = dc[q]; acc_n = 1; acc_f = df[q];
            }
        }
        const int c0 = __shfl_sync(0xffffffffu, acc_c, 0);
        const bool uni = !split && acc_c == c0 && acc_c >= 0;
        if (__all_sync(0xffffffffu, uni)) {
            const unsigned nw = __reduce_add_sync(0xffffffffu, acc_n);
            const unsigned hi = __reduce_add_sync(0xffffffffu, (unsigned)(acc_f >> 16));
            const unsigned lo = __reduce_add_sync(0xffffffffu, (unsigned)(acc_f & 0xFFFFull));
            if (lane == 0) hist_run(hist, c0, nw, ((unsigned long long)hi << 16) + lo);
        } else if (acc_c >= 0) {
            hist_run(hist, acc_c, acc_n, acc_f);
        }
        // queue the chunk's clock ends (slot order within the warp), run full batches
        if (QCAP > 0) {
            if (__any_sync(0xffffffffu, needm != 0u)) {        // warp-uniform; rare where collisions are
                unsigned m[CH];
#pragma unroll
                for (int q = 0; q < CH; ++q) m[q] = __ballot_sync(0xffffffffu, (needm >> q) & 1u);
                __syncwarp();                           // the last run's reads before new entries
                const unsigned lt = (1u << lane) - 1u;
#pragma unroll
                for (int q = 0; q < CH; ++q) {
                    if ((needm >> q) & 1u) Q[qn + __popc(m[q] & lt)] = (e0 + (unsigned)q) | (((candm >> q) & 1u) << 31);
                    qn += __popc(m[q]);
                }
                while (qn >= 32) {
                    qn -= 32;
                    __syncwarp();                       // the entries and the chunk's stores first
                    run_queue(qn + lane, true);
                }
            }
        }
    }
    if (QCAP > 0 && qn > 0) {                           // the rest of the queue
        __syncwarp();
        run_queue(lane, lane < qn);
    }
    if (KCAP > 0 && kn > 0) {                           // the rest of the ionizations
        __syncwarp();
        run_children(lane, lane < kn);
    }
    if (apcap != 0u) append_flush(P, ab, sh, half_e, half_i);
    if (n_stages > 0) {
        __syncthreads();
        if (sh.tile_abort) {
            // a tile never arrived (kErrTimeout raised): the item is abandoned
            // and the CTA streams no more tiles; wait, bounded, for every
            // buffer's last copy once
            if (tid == 0)
                for (int j = 0; j < n_stages; ++j) mbar_wait_bounded(&sh.full[j], ctrl, (tile_phase >> j) & 1u, 0u);
            return;
        }
    }
    // CTA epilogue: event counts (warp sums, one shared atomic per warp), histogram
    {
        unsigned vals[11] = {ev.cand, ev.coll[0], ev.coll[1], ev.coll[2], ev.coll[3], ev.iz,
                             ev.absorbed[0], ev.absorbed[1], ev.see, ev.see0, ev.renew};
#pragma unroll
        for (int k = 0; k < (AXIAL ? 11 : 10); ++k) {
            const unsigned w = __reduce_add_sync(0xffffffffu, vals[k]);
            if (lane == 0 && w) {
                if (k < 6) atomicAdd(&s_cnt[k], w);
                else if (k < 8) atomicAdd(&s_abs[k - 6], w);
                else if (k == 8) atomicAdd(&sh.s_see, w);
                else if (k == 9) atomicAdd(&sh.s_see0, w);
                else atomicAdd(&sh.s_renew, w);
            }
        }
    }
    hist_flush(hist, N, R_cta);
    if (diag) {
        const int nn = P.n_nodes;
        for (int j = tid; j <= N; j += blockDim.x) {
            const float h = hen[j];
            if (h != 0.0f) {
                const int jj = (PERIODIC && j == N) ? 0 : j;
                const double iv = (!PERIODIC && (jj == 0 || jj == N)) ? 1.0 / P.vol_wall : 1.0 / P.vol_interior;
                atomicAdd(&P.en_sum[SP * nn + jj], S.w * (double)h * iv);
            }
        }
        if (SP == 0)
            for (int j = tid; j < kEepfBins; j += blockDim.x)
                if (heepf[j]) atomicAdd(&P.eepf[j], (unsigned long long)heepf[j]);
        // block reductions of the kinetic-energy and J.E sums
        for (int o = 16; o > 0; o >>= 1) {
            ke_acc += __shfl_xor_sync(0xffffffffu, ke_acc, o);
            pw_acc += __shfl_xor_sync(0xffffffffu, pw_acc, o);
        }
        if (lane == 0) { sh.s_red[0][warp] = ke_acc; sh.s_red[1][warp] = pw_acc; }
        __syncthreads();
        if (tid == 0) {
            double ke = 0, pw = 0;
            for (int w = 0; w < (int)(blockDim.x / 32); ++w) { ke += sh.s_red[0][w]; pw += sh.s_red[1][w]; }
            atomicAdd(&P.ke_sum[SP], 0.5 * S.m * S.w * ke);
            atomicAdd(&P.pw_sum[SP], S.q * S.w * pw);
        }
    }
    if (tid == 0) {
        if (s_abs[0]) { atomicAdd(&ctrl->absorbed[SP][0], (unsigned long long)s_abs[0]); }
        if (s_abs[1]) { atomicAdd(&ctrl->absorbed[SP][1], (unsigned long long)s_abs[1]); }
        if (s_abs[0] + s_abs[1]) atomicAdd(&ctrl->n_dead[SP], (unsigned long long)(s_abs[0] + s_abs[1]));
        if (P.circuit && s_abs[0]) atomicAdd(&ctrl->st_abs0[SP], (unsigned long long)s_abs[0]);
        if (P.circuit && sh.s_see0) atomicAdd(&ctrl->st_see0, (unsigned long long)sh.s_see0);
        if (AXIAL && sh.s_renew) atomicAdd(&ctrl->renewed[SP], (unsigned long long)sh.s_renew);
        if (sh.s_see) atomicAdd(&ctrl->see, (unsigned long long)sh.s_see);
        if (s_cnt[0]) atomicAdd(&ctrl->cand[SP], (unsigned long long)s_cnt[0]);
        for (int k = 0; k < kMaxProc; ++k)
            if (s_cnt[1 + k]) atomicAdd(&ctrl->coll[SP][k], (unsigned long long)s_cnt[1 + k]);
        if (s_cnt[1 + kMaxProc]) atomicAdd(&ctrl->iz, (unsigned long long)s_cnt[1 + kMaxProc]);
    }
    __syncthreads();                                    // shared state free for the next item
}

// One case: CTA b takes the b-th of gridDim.x slices of the species.
// Launch chain of a step (programmatic dependent launches): the electron
// kernel waits for the previous field solve, then lets the ion kernel launch;
// the ion kernel reads nothing the electron kernel writes (each species
// processes its own first n_active slots, appends go beyond them, deposits
// and counters are atomic), so it runs into the electron kernel's tail and
// waits for it only before exiting, which keeps the field solve (launched
// after it, waiting for it) behind both.
template <int SP, bool PERIODIC, int MCC, bool STAGED, bool AXIAL>
// launch bounds: up to 1024 threads, 64 registers (two 512-thread or four
// 256-thread CTAs per SM when shared memory allows)
__global__ void __launch_bounds__(kStepThreads, 1) k_particle_step(const __grid_constant__ StepConst P)
{
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ StepShared sh;
    if (threadIdx.x == 0) {
        mbar_init(&sh.mbar, 1);
        for (int b = 0; b < kMaxStages; ++b) { mbar_init(&sh.full[b], 1); sh.tile_rel[b] = 0u; }
        sh.tile_abort = 0u;
    }
    __syncthreads();
    if (SP == 0) {
        grid_dep_wait();
        grid_dep_launch();
    }
    unsigned parity = 0, tile_phase = 0;
    particle_item<SP, PERIODIC, MCC, STAGED, AXIAL>(P, P.push, smem, sh, parity, tile_phase, blockIdx.x, gridDim.x);
    if (SP == 1) {
        grid_dep_launch();
        grid_dep_wait();
    }
}

// Launch shapes of the batch kernel, chosen per batch by its autotuner:
//   0: 512-thread CTAs, one per SM, up to 128 registers a thread, chunks of
//      one particle with three in flight per thread;
//   1: 512-thread CTAs, two per SM (64 registers), chunks of two, one ahead;
//   2: 1024-thread CTAs, one per SM (64 registers), chunks of two, one ahead
//      (the single-case kernels' shape);
//   3: 640-thread CTAs, one per SM (96 registers), chunks of two, one ahead.
template <int SHAPE> struct BatchShape;
template <> struct BatchShape<0> { static constexpr int threads = 512, minb = 1, chunk = 1, depth = 3; };
template <> struct BatchShape<1> { static constexpr int threads = 512, minb = 2, chunk = 2, depth = 1; };
template <> struct BatchShape<2> { static constexpr int threads = 1024, minb = 1, chunk = 2, depth = 1; };
template <> struct BatchShape<3> { static constexpr int threads = 640, minb = 1, chunk = 2, depth = 1; };
// 0-3: the persistent kernel; 4, 5: the grid of work items (k_batch_grid) in
// the launch shapes of 2 (1024 threads) and 3 (640 threads)
constexpr int kBatchShapes = 6;

// Out-of-line item for the batch kernel: each species' body keeps its own
// register allocation instead of the union of both.
template <int SP, bool PERIODIC, int MCC, bool STAGED, int SHAPE>
__device__ __noinline__ void particle_item_call(const StepConst &P, unsigned char *smem, StepShared &sh,
                                               unsigned &parity, unsigned &tile_phase, long long k_item,
                                               long long n_items)
{
    particle_item<SP, PERIODIC, MCC, STAGED, false, BatchShape<SHAPE>::chunk, BatchShape<SHAPE>::depth>(
        P, P.push, smem, sh, parity, tile_phase, k_item, n_items);
}

// Many cases in one persistent launch: CTAs take (case, species, slice) work
// items from an atomic counter (reset by the batched field solve).
struct BatchItem {
    int case_idx, species, k, nk;
};

template <bool PERIODIC, int MCC0, int MCC1, bool STAGED, int SHAPE>
__global__ void __launch_bounds__(BatchShape<SHAPE>::threads, BatchShape<SHAPE>::minb)
    k_batch_particle_step(const StepConst *__restrict__ cases, const BatchItem *__restrict__ items, int n_items,
                          unsigned *next_item)
{
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ StepShared sh;
    __shared__ int s_item[2];
    __shared__ StepConst sP;                            // the item's case constants (read like parameters)
    if (threadIdx.x == 0) {
        mbar_init(&sh.mbar, 1);
        for (int b = 0; b < kMaxStages; ++b) { mbar_init(&sh.full[b], 1); sh.tile_rel[b] = 0u; }
        sh.tile_abort = 0u;
    }
    if (threadIdx.x == 0) s_item[0] = (int)atomicAdd(next_item, 1u);
    __syncthreads();
    unsigned parity = 0, tile_phase = 0;
    int cur_case = -1;
    // The next item's index is taken while this one runs (two slots: the
    // barrier that ends an item orders every read of one slot before thread 0
    // writes it again).
    for (int k = 0;; ++k) {
        const int it = s_item[k & 1];
        if (it >= n_items) break;
        if (threadIdx.x == 0) s_item[(k + 1) & 1] = (int)atomicAdd(next_item, 1u);
        const BatchItem w = items[it];
        if (w.case_idx != cur_case) {                   // copy the case's constants into shared memory
            const int *src = reinterpret_cast<const int *>(&cases[w.case_idx]);
            int *dst = reinterpret_cast<int *>(&sP);
            for (int j = threadIdx.x; j < (int)(sizeof(StepConst) / sizeof(int)); j += blockDim.x) dst[j] = src[j];
            cur_case = w.case_idx;
            __syncthreads();
        }
        if (w.species == 0)
            particle_item_call<0, PERIODIC, MCC0, STAGED, SHAPE>(sP, smem, sh, parity, tile_phase, w.k, w.nk);
        else
            particle_item_call<1, PERIODIC, MCC1, STAGED, SHAPE>(sP, smem, sh, parity, tile_phase, w.k, w.nk);
        __syncthreads();                                // s_item[(k + 1) & 1] written
    }
}

// Batched step as a grid of work items, one CTA each, for up to kGridCases
// cases per launch.  The item list and every case's push constants travel in
// the kernel parameter: a CTA's item comes from the parameter at blockIdx.x,
// the same for all its threads, so the particle loop reads its case's push
// constants from the constant bank, as the single-case kernel reads its own,
// instead of from shared memory (where they cost an instruction and a
// register each, and every shared store or atomic of the loop forces a
// reload).  The other case constants are copied into shared memory once.
// Items are listed largest first, and the block scheduler hands them to SMs
// as they free up.
constexpr int kGridCases = 256;
constexpr int kGridItems = 1536;
struct GridTable {
    uint32_t item[kGridItems];          // case | k << 8 | nk << 19 (k, nk < 2048)
    CasePush push[kGridCases];
};
static_assert(sizeof(GridTable) <= 32764, "a kernel parameter holds at most 32764 bytes");

// One launch per species and table, chained by programmatic dependent
// launches: a launch lets the next one start as its last CTAs start (the next
// needs nothing it writes: each species processes its own first n_active
// slots, appends go beyond them, deposits and counters are atomic) and waits
// for the previous one before it exits, so that the last launch of a step
// ends after all of them.
template <int SP, bool PERIODIC, int MCC, int SHAPE>
__global__ void __launch_bounds__(BatchShape<SHAPE>::threads, BatchShape<SHAPE>::minb)
    k_batch_grid(const __grid_constant__ GridTable T, const StepConst *__restrict__ cases, int case0)
{
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ StepShared sh;
    __shared__ StepConst sP;
    grid_dep_launch();
    const uint32_t w = T.item[blockIdx.x];
    const int ci = (int)(w & 0xFFu);
    const long long k = (long long)((w >> 8) & 0x7FFu), nk = (long long)(w >> 19);
    if (threadIdx.x == 0) {
        mbar_init(&sh.mbar, 1);
        for (int b = 0; b < kMaxStages; ++b) { mbar_init(&sh.full[b], 1); sh.tile_rel[b] = 0u; }
        sh.tile_abort = 0u;
    }
    {
        const int *src = reinterpret_cast<const int *>(&cases[case0 + ci]);
        int *dst = reinterpret_cast<int *>(&sP);
        for (int j = threadIdx.x; j < (int)(sizeof(StepConst) / sizeof(int)); j += blockDim.x) dst[j] = src[j];
    }
    __syncthreads();
    unsigned parity = 0, tile_phase = 0;
    particle_item<SP, PERIODIC, MCC, false, false, BatchShape<SHAPE>::chunk, BatchShape<SHAPE>::depth>(
        sP, T.push[ci], smem, sh, parity, tile_phase, k, nk);
    grid_dep_wait();
}

// Leapfrog start: v(0) -> v(-dt/2) by a Boris step of -dt/2 in E^0.
template <int SP>
__global__ void k_rewind(const __grid_constant__ StepConst P)
{
    const SpPush &S = P.push.sp[SP];
    const SpeciesBufs B = P.buf[SP][P.ctrl->cur[SP]];
    const long long n = (long long)P.ctrl->n_active[SP];
    // half-step constants: a = q(-dt/2)/(2m) = -c_e/2; t = a B; s = 2t/(1+t^2)
    const float a = -0.5f * S.c_e;
    const float t0 = -0.5f * S.tB[0] / 1.0f, t1 = -0.5f * S.tB[1], t2 = -0.5f * S.tB[2];
    const float tt = t0 * t0 + t1 * t1 + t2 * t2;
    const float s0 = 2.0f * t0 / (1.0f + tt), s1 = 2.0f * t1 / (1.0f + tt), s2 = 2.0f * t2 / (1.0f + tt);
    const float ey = S.cEy * -0.5f, ez = S.cEz * -0.5f;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const int raw = B.cell[i];
        if (raw < 0) continue;
        const int c = raw & kCellMask;
        const float o = B.off[i];
        const float2 ep = P.E32p[c];
        const float ex = (1.0f - o) * ep.x + o * ep.y + P.push.ex_ext;
        const float hx = a * ex;
        const float3 vm = make_float3(B.vx[i] + hx, B.vy[i] + ey, B.vz[i] + ez);
        const float3 vp = make_float3(vm.x + (vm.y * t2 - vm.z * t1), vm.y + (vm.z * t0 - vm.x * t2),
                                      vm.z + (vm.x * t1 - vm.y * t0));
        B.vx[i] = vm.x + (vp.y * s2 - vp.z * s1) + hx;
        B.vy[i] = vm.y + (vp.z * s0 - vp.x * s2) + ey;
        B.vz[i] = vm.z + (vp.x * s1 - vp.y * s0) + ez;
    }
}

// Particle loader: n particles of species sp sampled from node profiles.
// Particle k has id = id_base + k and draws Philox counter
// (id, 0xFFFFFFFF, sp << 16 | 0x100 + j, 1), j = 0, 1.  The cell is the j with
// cdf[j] <= u < cdf[j+1] (FP64, cdf = cumulative CIC mass of the linear
// density); the offset inverts the linear density inside the cell,
// delta = u' (a+b) / (a + sqrt(a^2 + u' (b^2 - a^2))) with a, b the node
// densities; the velocity is Maxwellian at the linearly interpolated
// temperature plus a drift.
__global__ void k_load_profile(SpeciesBufs B, long long n, int N, const double *__restrict__ cdf,
                               const float *__restrict__ dens, const float *__restrict__ temp_ev, float vt_per_sqrt_ev,
                               float drift_x, float drift_y, float drift_z, uint32_t id_base, int sp, uint32_t k0,
                               uint32_t k1)
{
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x) {
        const uint32_t id = id_base + (uint32_t)k;
        const uint4 r = philox4x32_10(make_uint4(id, 0xFFFFFFFFu, ((uint32_t)sp << 16) | 0x100u, 1u), k0, k1);
        const uint4 r2 = philox4x32_10(make_uint4(id, 0xFFFFFFFFu, ((uint32_t)sp << 16) | 0x101u, 1u), k0, k1);
        const double u = (double)u01(r.x);
        int lo = 0, hi = N;                                  // cdf[lo] <= u < cdf[hi]
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (cdf[mid] <= u) lo = mid; else hi = mid;
        }
        const float a = dens[lo], b = dens[lo + 1], u2 = u01(r.y);
        const float den = a + sqrtf(fmaxf(a * a + u2 * (b * b - a * a), 0.0f));
        float o = den > 0.0f ? u2 * (a + b) / den : u2;
        o = fminf(fmaxf(o, 0.0f), 0.99999994f);
        const float T = (1.0f - o) * temp_ev[lo] + o * temp_ev[lo + 1];
        const float vt = vt_per_sqrt_ev * sqrtf(fmaxf(T, 0.0f));
        const float2 g01 = box_muller(u01(r.z), u01(r.w));
        const float2 g23 = box_muller(u01(r2.x), u01(r2.y));
        B.cell[k] = lo;
        B.off[k] = o;
        B.vx[k] = fmaf(vt, g01.x, drift_x);
        B.vy[k] = fmaf(vt, g01.y, drift_y);
        B.vz[k] = fmaf(vt, g23.x, drift_z);
        B.id[k] = id;
        if (B.z) B.z[k] = 0.0f;
    }
}

// Deposit of all particles of a species (the state at load), validation of
// the loaded cells/offsets (plain cell indices: a load starts every species'
// clocks afresh), and each particle's first collision clock.
__global__ void __launch_bounds__(256) k_deposit_species(const __grid_constant__ StepConst P, int sp)
{
    // the particles of a CTA's contiguous chunk go into a shared histogram
    // (count, sum of f >> 16, sum of f & 0xFFFF per cell; 12 N bytes), flushed
    // to the raw deposit after every kDepositSpan particles, so that no counter
    // overflows and each cell costs two global atomics a flush instead of two
    // a particle
    extern __shared__ unsigned dsm[];
    const SpeciesBufs B = P.buf[sp][P.ctrl->cur[sp]];
    const long long n = (long long)P.ctrl->n_active[sp];
    const int N = P.n_cells;
    const uint32_t step = (uint32_t)P.ctrl->step;
    unsigned *cnt = dsm, *fhi = dsm + N, *flo = dsm + 2 * N;
    for (int j = threadIdx.x; j < 3 * N; j += blockDim.x) dsm[j] = 0u;
    const long long chunk = (n + gridDim.x - 1) / gridDim.x;
    const long long lo = min((long long)blockIdx.x * chunk, n), hi = min(lo + chunk, n);
    unsigned long long *R = P.R[sp] + (size_t)(blockIdx.x % kDepositCopies) * P.r_stride;
    for (long long s0 = lo; s0 < hi; s0 += kDepositSpan) {
        __syncthreads();                                // counters zero
        const long long s1 = min(s0 + (long long)kDepositSpan, hi);
        for (long long i = s0 + threadIdx.x; i < s1; i += blockDim.x) {
            const int c = B.cell[i];
            const float o = B.off[i];
            if (c < 0) continue;
            if (c >= N || !(o >= 0.0f && o < 1.0f)) { atomicOr(&P.ctrl->err, kErrLoad); B.cell[i] = -1; continue; }
            if (P.push.sp[sp].lam > 0.0f) B.cell[i] = c | (int)(first_clock(P, sp, B.id[i], step) << kCellBits);
            const uint32_t f = __float2uint_rz(o * 4294967296.0f);
            atomicAdd(&cnt[c], 1u);
            atomicAdd(&fhi[c], f >> 16);
            atomicAdd(&flo[c], f & 0xFFFFu);
        }
        __syncthreads();
        for (int c = threadIdx.x; c < N; c += blockDim.x) {
            const unsigned k = cnt[c];
            if (k == 0u) continue;
            const unsigned long long F = ((unsigned long long)fhi[c] << 16) + flo[c];
            const int c1 = (P.periodic && c + 1 == N) ? 0 : c + 1;
            atomicAdd(&R[c], ((unsigned long long)k << 32) - F);
            atomicAdd(&R[c1], F);
            cnt[c] = 0u; fhi[c] = 0u; flo[c] = 0u;
        }
    }
}

} // namespace pic
