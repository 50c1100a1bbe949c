// field_sort.cuh -- FP64 field solve (one CTA) and the counting sort by cell.
#pragma once
#include "pic_device.cuh"
#include <cooperative_groups.h>

namespace pic {

// In-place inclusive scan of a[0..M) in shared memory by one CTA, in a fixed
// order (bit-identical on every run).  `warp_tot` needs blockDim/32 doubles.
__device__ void block_scan_inclusive(double *a, int M, double *warp_tot)
{
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
    const int k = (M + blockDim.x - 1) / blockDim.x;
    const int lo = min(tid * k, M), hi = min(lo + k, M);
    double s = 0.0;
    for (int i = lo; i < hi; ++i) s += a[i];
    double incl = s;
    for (int o = 1; o < 32; o <<= 1) {
        const double y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    if (lane == 31) warp_tot[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        double w = lane < nw ? warp_tot[lane] : 0.0;
        for (int o = 1; o < 32; o <<= 1) {
            const double y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        if (lane < nw) warp_tot[lane] = w;
    }
    __syncthreads();
    double run = (incl - s) + (warp > 0 ? warp_tot[warp - 1] : 0.0);
    __syncthreads();
    for (int i = lo; i < hi; ++i) { run += a[i]; a[i] = run; }
    __syncthreads();
}

// Sum of v over the CTA (fixed order), result broadcast to every thread.
__device__ double block_sum(double v, double *red)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    __syncthreads();
    if (lane == 0) red[warp] = v;
    __syncthreads();
    double t = 0.0;
    for (int w = 0; w < nw; ++w) t += red[w];
    __syncthreads();
    return t;
}

// Exclusive prefix of one 64-bit integer per thread over the CTA (exact).
__device__ unsigned long long block_exclusive_u64(unsigned long long v, unsigned long long *red,
                                                  unsigned long long *total)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    unsigned long long incl = v;
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    __syncthreads();
    if (lane == 31) red[warp] = incl;
    __syncthreads();
    unsigned long long off = 0, tot = 0;
    for (int w = 0; w < nw; ++w) {
        if (w < warp) off += red[w];
        tot += red[w];
    }
    *total = tot;
    return off + incl - v;
}

// Exclusive prefix of one FP64 value per thread over the CTA (fixed order).
__device__ double block_exclusive_f64(double v, double *red, double *total)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    double incl = v;
    for (int o = 1; o < 32; o <<= 1) {
        const double y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    __syncthreads();
    if (lane == 31) red[warp] = incl;
    __syncthreads();
    double off = 0.0, tot = 0.0;
    for (int w = 0; w < nw; ++w) {
        if (w < warp) off += red[w];
        tot += red[w];
    }
    *total = tot;
    return off + (incl - v);
}

// Poisson's equation (paper §1) and the node field, FP64, on a cluster of
// kFieldCluster CTAs (one SM each) that exchange partial sums through
// distributed shared memory.
// (phi_{i-1} - 2 phi_i + phi_{i+1}) / dx^2 = -rho_i / eps0 on the interior
// nodes; bounded: phi_0 = V(t), phi_N = 0; periodic: neutralised rho, phi_0 = 0
// on the N-1 interior equations (the one at node 0 then holds), mean of phi
// removed.  With r_k = rho_k dx^2/eps0, S_m = sum_{k=1..m} r_k and
// T_i = sum_{m<i} S_m, the difference equation integrates exactly to
//   phi_i = phi_0 + i d_0 - T_i,   d_0 = (T_N - phi_0) / N.
// The charge enters as exact integer prefix sums of the fixed-point deposits,
// P_s[m] = sum_{k=1..m} R_s[k], so S_m = sum_s c_s P_s[m] + b m with
// c_s = (dx/eps0) q_s w_s 2^-32 and b the uniform part; only the second sum
// and the per-node potential, field and energy use FP64.  B300's FP64 rate is
// low, so the nodes are split over the cluster's SMs and no division is done
// per node.  Partial sums are combined in rank order (bit-identical runs).
// E: central differences inside; Gauss's law over the half cell at an
// electrode; wrap-around when periodic.
// mode 0: field of the loaded state at t = 0; mode 1: end of a step
// (t = (step+1) dt, moments accumulated, counters advanced).
__global__ void __cluster_dims__(kFieldCluster, 1, 1) __launch_bounds__(kFieldThreads)
    k_field(const __grid_constant__ StepConst P, int mode, unsigned long long *R_last)
{
    namespace cg = cooperative_groups;
    cg::cluster_group cl = cg::this_cluster();
    extern __shared__ __align__(16) double fsm[];
    __shared__ unsigned long long ured[kFieldThreads / 32];
    __shared__ double red[kFieldThreads / 32];
    __shared__ unsigned long long x_seg[2], x_tot[2];   // published CTA totals (integer charge)
    __shared__ double x_S, x_phi, x_fe, s_bcast[2];
    __shared__ unsigned long long s_off[2], s_all[2];
    __shared__ int x_bad;
    const int rank = (int)cl.block_rank();
    const int N = P.n_cells, nn = P.n_nodes, tid = threadIdx.x, ns = P.n_species;
    const int per_cta = (N + 1 + kFieldCluster - 1) / kFieldCluster;
    const int c_lo = min(rank * per_cta, N + 1), c_hi = min(c_lo + per_cta, N + 1);
    const int per = (c_hi - c_lo + blockDim.x - 1) / blockDim.x;
    const int lo = min(c_lo + tid * per, c_hi), hi = min(lo + per, c_hi);
    double *phi = fsm;                                                   // [per_cta], local index i - c_lo
    double *T = fsm + per_cta;                                           // [per_cta]
    unsigned long long *Ps = reinterpret_cast<unsigned long long *>(fsm + 2 * per_cta);   // [2][per_cta]
    Ctrl *ctrl = P.ctrl;
    const long long step = ctrl->step;
    const bool diag = mode == 1 && P.diag_interval > 0 && ((step + 1) % P.diag_interval) == 0;

    // 1. raw deposits (periodic: node N folds onto node 0), integer moment sums
    unsigned long long tot_s[2] = {0ull, 0ull}, seg_s[2] = {0ull, 0ull};
    for (int s = 0; s < ns; ++s)
        for (int i = lo; i < hi; ++i) {
            unsigned long long r = 0ull;
            if (i < nn) {
                r = P.R[s][i];
                if (P.periodic && i == 0) r += P.R[s][N];
                R_last[s * nn + i] = r;
                if (mode == 1) {
                    P.Rsum[s * nn + i] += r;
                    if (diag) P.Rdiag[s * nn + i] += r;
                }
                tot_s[s] += r;
            }
            Ps[s * per_cta + (i - c_lo)] = r;
            if (i >= 1 && i <= N - 1) seg_s[s] += r;
        }
    unsigned long long run_s[2] = {0ull, 0ull};
    for (int s = 0; s < ns; ++s) {
        unsigned long long t1, t2;
        run_s[s] = block_exclusive_u64(seg_s[s], ured, &t1);
        (void)block_exclusive_u64(tot_s[s], ured, &t2);
        if (tid == 0) { x_seg[s] = t1; x_tot[s] = t2; }
    }
    cl.sync();                                                           // totals published; R fully read
    // warp 0: lane r reads rank r's totals (parallel remote reads), combines them
    if (tid < 32) {
        const int lane = tid;
        for (int s = 0; s < ns; ++s) {
            const unsigned long long vs = lane < kFieldCluster ? cl.map_shared_rank(x_seg, lane)[s] : 0ull;
            const unsigned long long vt = lane < kFieldCluster ? cl.map_shared_rank(x_tot, lane)[s] : 0ull;
            unsigned long long below = lane < rank ? vs : 0ull, all = vt;
            for (int o = 16; o > 0; o >>= 1) {
                below += __shfl_xor_sync(0xffffffffu, below, o);
                all += __shfl_xor_sync(0xffffffffu, all, o);
            }
            if (lane == 0) { s_off[s] = below; s_all[s] = all; }
        }
    }
    __syncthreads();
    unsigned long long all_s[2] = {0ull, 0ull};
    for (int s = 0; s < ns; ++s) {
        run_s[s] += s_off[s];
        all_s[s] = s_all[s];
        for (int i = lo; i < hi; ++i) {
            if (i >= 1 && i <= N - 1) run_s[s] += Ps[s * per_cta + (i - c_lo)];
            Ps[s * per_cta + (i - c_lo)] = run_s[s];                    // P_s[i], P_s[0] = 0
        }
        for (int i = lo; i < hi; ++i) P.R[s][i] = 0ull;
    }
    // 2. S_m = sum_s c_s P_s[m] + b m;  T_i = sum_{m<i} S_m
    double b = P.bg_r;
    if (P.periodic) {
        double q = 0.0;
        for (int s = 0; s < ns; ++s) q += P.cq[s] * (double)(long long)all_s[s];
        b = -q / N;                                                      // neutralising part (bg cancels)
    }
    double segS = 0.0;
    for (int i = lo; i < hi; ++i) {
        double S = 0.0;
        if (i < N) {
            S = b * (double)i;
            for (int s = 0; s < ns; ++s) S = fma(P.cq[s], (double)(long long)Ps[s * per_cta + (i - c_lo)], S);
        }
        T[i - c_lo] = S;
        segS += S;
    }
    double ctaS;
    double runT = block_exclusive_f64(segS, red, &ctaS);
    if (tid == 0) x_S = ctaS;
    cl.sync();
    if (tid < 32) {                                                      // ranks' S totals, fixed order
        double v = tid < kFieldCluster ? *cl.map_shared_rank(&x_S, tid) : 0.0;
        double below = 0.0, all = 0.0;
        for (int r = 0; r < kFieldCluster; ++r) {
            const double y = __shfl_sync(0xffffffffu, v, r);
            if (r < rank) below += y;
            all += y;
        }
        if (tid == 0) { s_bcast[0] = below; s_bcast[1] = all; }
    }
    __syncthreads();
    runT += s_bcast[0];
    const double totS = s_bcast[1];
    __syncthreads();
    for (int i = lo; i < hi; ++i) {
        const double S = T[i - c_lo];
        T[i - c_lo] = runT;                                              // T_i
        runT += S;
    }
    if (tid == 0) {
        double phi0 = 0.0;
        if (!P.periodic) {
            const double t = mode == 0 ? 0.0 : (double)(step + 1) * P.dt;
            for (int h = 0; h < P.n_harm; ++h) phi0 += P.harm_a[h] * cos(2.0 * M_PI * P.harm_f[h] * t + P.harm_p[h]);
        }
        s_bcast[0] = phi0;
        s_bcast[1] = (totS - phi0) / N;                                  // d_0 (T_N = sum of all S)
    }
    __syncthreads();
    const double phi0 = s_bcast[0], d0 = s_bcast[1];
    double segT = 0.0;
    for (int i = lo; i < hi; ++i) {
        double v = fma((double)i, d0, phi0) - T[i - c_lo];
        if (!P.periodic && i == N) v = 0.0;
        phi[i - c_lo] = v;
        if (i < N) segT += v;
    }
    if (P.periodic) {
        double ctaT;
        (void)block_exclusive_f64(segT, red, &ctaT);
        if (tid == 0) x_phi = ctaT;
        cl.sync();
        if (tid < 32) {
            double v = tid < kFieldCluster ? *cl.map_shared_rank(&x_phi, tid) : 0.0;
            double all = 0.0;
            for (int r = 0; r < kFieldCluster; ++r) all += __shfl_sync(0xffffffffu, v, r);
            if (tid == 0) s_bcast[0] = all;
        }
        __syncthreads();
        const double pm = s_bcast[0] / N;
        for (int i = lo; i < hi; ++i) phi[i - c_lo] -= pm;
    }
    cl.sync();                                                           // every phi final and visible
    // 3. node field (neighbours of the slice ends come from the owning CTA)
    auto phi_at = [&](int j) -> double {
        const int owner = j / per_cta;
        if (owner == rank) return phi[j - c_lo];
        return cl.map_shared_rank(phi, owner)[j - owner * per_cta];
    };
    double fe = 0.0;
    int bad = 0;
    for (int i = lo; i < hi && i < nn; ++i) {
        double E;
        const double ph = phi[i - c_lo];
        if (P.periodic) {
            const int ip = i + 1 == N ? 0 : i + 1, im = i == 0 ? N - 1 : i - 1;
            E = (phi_at(im) - phi_at(ip)) * P.inv_2dx;
            fe = fma(E, E, fe);
        } else if (i == 0 || i == N) {
            double rq = P.bg_charge;                                     // charge density of the wall node
            for (int s = 0; s < ns; ++s) rq = fma(P.rho_wall[s], (double)(long long)R_last[s * nn + i], rq);
            E = i == 0 ? (ph - phi_at(1)) * P.inv_dx - rq * P.half_dx_eps0
                       : (phi_at(N - 1) - ph) * P.inv_dx + rq * P.half_dx_eps0;
            fe = fma(0.5 * E, E, fe);
        } else {
            E = (phi_at(i - 1) - phi_at(i + 1)) * P.inv_2dx;
            fe = fma(E, E, fe);
        }
        P.E[i] = E;
        P.phi[i] = ph;
        P.E32[i] = (float)E;
        if (P.periodic && i == 0) P.E32[N] = (float)E;
        if (mode == 1) P.phi_sum[i] += ph;
        bad |= !isfinite(ph) || !isfinite(E);
    }
    fe = block_sum(fe, red);
    bad = __syncthreads_or(bad);
    if (tid == 0) { x_fe = fe; x_bad = bad; }
    cl.sync();
    if (rank == 0 && tid < 32) {
        const double v = tid < kFieldCluster ? *cl.map_shared_rank(&x_fe, tid) : 0.0;
        const int bv = tid < kFieldCluster ? *cl.map_shared_rank(&x_bad, tid) : 0;
        double fe_all = 0.0;
        for (int r = 0; r < kFieldCluster; ++r) fe_all += __shfl_sync(0xffffffffu, v, r);
        const int bad_all = __any_sync(0xffffffffu, bv != 0);
        if (tid == 0) {
        if (bad_all) atomicOr(&ctrl->err, kErrNumeric);
        if (mode == 1) {
            P.fe_hist[ctrl->fe_n % (unsigned long long)P.fe_cap] = fe_all * P.fe_c;
            ctrl->fe_n += 1;
            ctrl->n_steps_acc += 1;
            if (diag) ctrl->n_diag_acc += 1;
            for (int s = 0; s < ns; ++s) {
                unsigned long long nt = ctrl->n_total[s];
                if (nt > P.cap[s]) nt = P.cap[s];
                ctrl->n_total[s] = nt;
                ctrl->n_active[s] = nt;
            }
            ctrl->step = step + 1;
        }
        }
    }
    cl.sync();                                                           // no CTA leaves while read remotely
}

// ---------------------------------------------------------------------------
// Counting sort by cell (also drops absorbed slots: cell outside [0, N)):
// count -> exclusive scan -> scatter into the other half.  The same kernels
// serve a case (halves = its ping-pong storage, count and current half read on
// the device) and the stand-alone entry point (halves = caller's in/out).
// ---------------------------------------------------------------------------
struct SortHalves {
    SpeciesBufs h[2];
};

__device__ __forceinline__ long long sort_count_of(const unsigned long long *n_dev, long long n_host)
{
    return n_dev ? (long long)*n_dev : n_host;
}

__global__ void k_cells_count(SortHalves H, const int32_t *cur_dev, const unsigned long long *n_dev, long long n_host,
                              int N, unsigned *counts)
{
    extern __shared__ unsigned cnt_s[];
    for (int j = threadIdx.x; j < N; j += blockDim.x) cnt_s[j] = 0u;
    __syncthreads();
    const SpeciesBufs A = H.h[cur_dev ? *cur_dev : 0];
    const long long n = sort_count_of(n_dev, n_host);
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const int c = A.cell[i];
        if (c >= 0 && c < N) atomicAdd(&cnt_s[c], 1u);
    }
    __syncthreads();
    for (int j = threadIdx.x; j < N; j += blockDim.x)
        if (cnt_s[j]) atomicAdd(&counts[j], cnt_s[j]);
}

// cursor[j] = sum_{k<j} counts[k]; cursor[N] = total (one CTA, exact: counts < 2^53)
__global__ void __launch_bounds__(1024) k_cells_scan(const unsigned *counts, int N, unsigned long long *cursor)
{
    extern __shared__ __align__(16) double ssm[];
    __shared__ double red[32];
    for (int j = threadIdx.x; j < N; j += blockDim.x) ssm[j] = (double)counts[j];
    __syncthreads();
    block_scan_inclusive(ssm, N, red);
    for (int j = threadIdx.x; j < N; j += blockDim.x) cursor[j] = (unsigned long long)(ssm[j] - (double)counts[j]);
    if (threadIdx.x == 0) cursor[N] = (unsigned long long)ssm[N - 1];
}

constexpr int kSortChunk = 8192;

// Each CTA reserves, per cell, one contiguous range for its chunk's particles
// (one global atomic per touched cell), then places them with shared atomics.
__global__ void k_cells_scatter(SortHalves H, const int32_t *cur_dev, const unsigned long long *n_dev, long long n_host,
                                int N, unsigned long long *cursor)
{
    extern __shared__ __align__(16) unsigned char xsm[];
    unsigned long long *base = reinterpret_cast<unsigned long long *>(xsm);
    unsigned *lcnt = reinterpret_cast<unsigned *>(xsm + 8 * (size_t)N);
    for (int j = threadIdx.x; j < N; j += blockDim.x) lcnt[j] = 0u;
    __syncthreads();
    const int half = cur_dev ? *cur_dev : 0;
    const SpeciesBufs A = H.h[half], D = H.h[half ^ 1];
    const long long n = sort_count_of(n_dev, n_host);
    const long long lo = (long long)blockIdx.x * kSortChunk, hi = min(lo + kSortChunk, n);
    for (long long i = lo + threadIdx.x; i < hi; i += blockDim.x) {
        const int c = A.cell[i];
        if (c >= 0 && c < N) atomicAdd(&lcnt[c], 1u);
    }
    __syncthreads();
    for (int j = threadIdx.x; j < N; j += blockDim.x) {
        const unsigned k = lcnt[j];
        base[j] = k ? atomicAdd(&cursor[j], (unsigned long long)k) : 0ull;
        lcnt[j] = 0u;
    }
    __syncthreads();
    for (long long i = lo + threadIdx.x; i < hi; i += blockDim.x) {
        const int c = A.cell[i];
        if (c < 0 || c >= N) continue;
        const unsigned long long p = base[c] + atomicAdd(&lcnt[c], 1u);
        D.cell[p] = c; D.off[p] = A.off[i]; D.vx[p] = A.vx[i]; D.vy[p] = A.vy[i]; D.vz[p] = A.vz[i];
        D.id[p] = A.id[i];
    }
}

// case epilogue: the sorted half becomes current; counts reset for next time
__global__ void k_sort_finish(const __grid_constant__ StepConst P, int sp, const unsigned long long *total)
{
    const int N = P.n_cells;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        Ctrl *ctrl = P.ctrl;
        const unsigned long long live = *total;
        ctrl->cur[sp] ^= 1;
        ctrl->n_total[sp] = live;
        ctrl->n_active[sp] = live;
        ctrl->n_dead[sp] = 0ull;
    }
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < N; j += gridDim.x * blockDim.x) P.sort_count[j] = 0u;
}

// ---------------------------------------------------------------------------
// Kernel-level entry points
// ---------------------------------------------------------------------------
__global__ void k_philox(uint32_t k0, uint32_t k1, long long n, const uint4 *ctr, uint4 *out)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        out[i] = philox4x32_10(ctr[i], k0, k1);
}

__global__ void k_deposit_plain(int N, int periodic, long long n, const int32_t *cell, const float *off,
                                unsigned long long *R)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const int c = cell[i];
        const float o = off[i];
        if (c < 0 || c >= N || !(o >= 0.0f && o < 1.0f)) continue;     // outside the grid: not deposited
        const uint32_t f = __float2uint_rz(o * 4294967296.0f);
        const int c1 = (periodic && c + 1 == N) ? 0 : c + 1;
        atomicAdd(&R[c], (1ull << 32) - f);
        atomicAdd(&R[c1], (unsigned long long)f);
    }
}

} // namespace pic
