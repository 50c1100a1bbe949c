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

typedef unsigned __int128 u128;

__device__ __forceinline__ u128 shfl_up_u128(u128 v, int o)
{
    const unsigned long long lo = __shfl_up_sync(0xffffffffu, (unsigned long long)v, o);
    const unsigned long long hi = __shfl_up_sync(0xffffffffu, (unsigned long long)(v >> 64), o);
    return ((u128)hi << 64) | lo;
}
__device__ __forceinline__ u128 shfl_u128(u128 v, int src)
{
    const unsigned long long lo = __shfl_sync(0xffffffffu, (unsigned long long)v, src);
    const unsigned long long hi = __shfl_sync(0xffffffffu, (unsigned long long)(v >> 64), src);
    return ((u128)hi << 64) | lo;
}
__device__ __forceinline__ double u128_to_double(u128 v)
{
    return fma((double)(unsigned long long)(v >> 64), 18446744073709551616.0, (double)(unsigned long long)v);
}
__device__ __forceinline__ bool finite_bits(double x)
{
    return ((unsigned long long)__double_as_longlong(x) & 0x7FF0000000000000ull) != 0x7FF0000000000000ull;
}

// Exclusive prefix over the CTA of NV integer values per thread (all summed
// together in one pass), exact.  Warp totals are scanned by warp 0.
template <typename T, int NV>
__device__ void block_exclusive_vec(const T (&v)[NV], T (&excl)[NV], T (&total)[NV], T (*red)[NV])
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    T incl[NV];
#pragma unroll
    for (int j = 0; j < NV; ++j) incl[j] = v[j];
    for (int o = 1; o < 32; o <<= 1) {
#pragma unroll
        for (int j = 0; j < NV; ++j) {
            T y;
            if constexpr (sizeof(T) == 16) y = shfl_up_u128(incl[j], o);
            else y = __shfl_up_sync(0xffffffffu, incl[j], o);
            if (lane >= o) incl[j] += y;
        }
    }
    __syncthreads();
    if (lane == 31)
#pragma unroll
        for (int j = 0; j < NV; ++j) red[warp][j] = incl[j];
    __syncthreads();
    if (warp == 0) {
#pragma unroll
        for (int j = 0; j < NV; ++j) {
            T w = lane < nw ? red[lane][j] : T(0);
            for (int o = 1; o < 32; o <<= 1) {
                T y;
                if constexpr (sizeof(T) == 16) y = shfl_up_u128(w, o);
                else y = __shfl_up_sync(0xffffffffu, w, o);
                if (lane >= o) w += y;
            }
            if (lane < nw) red[lane][j] = w;                        // inclusive over warps
        }
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < NV; ++j) {
        excl[j] = (warp > 0 ? red[warp - 1][j] : T(0)) + incl[j] - v[j];
        total[j] = red[nw - 1][j];
    }
    __syncthreads();
}

// Poisson's equation (paper §1) and the node field, on a cluster of CL CTAs
// (one SM each; CL a power of two, CL * kFieldThreads > n_cells), each owning
// a contiguous slice of nodes, one node per thread.
// (phi_{i-1} - 2 phi_i + phi_{i+1}) / dx^2 = -rho_i / eps0 on the interior
// nodes; bounded: phi_0 = V(t), phi_N = 0; periodic: neutralised rho, phi_0 = 0
// on the N-1 interior equations (the one at node 0 then holds), mean of phi
// removed.  With the fixed-point deposits R_s, their exact prefix sums
//   P_s[m] = sum_{k=1..m} R_s[k]   (u64),   Q_s[i] = sum_{m<i} P_s[m]   (u128),
// c_s = (dx/eps0) q_s w_s 2^-32 and b the uniform part of the source, the
// difference equation integrates exactly to
//   S_m = sum_s c_s P_s[m] + b m,   d_m = phi_{m+1} - phi_m = d_0 - S_m,
//   phi_i = phi_0 + i d_0 - T_i,    T_i = sum_s c_s Q_s[i] + b i(i-1)/2,
//   d_0 = (T_N - phi_0) / N,
// and the central-difference field is E_i = (S_i + S_{i-1} - 2 d_0) / (2dx)
// (Gauss's law over the half cell at an electrode: E_0 = -d_0/dx - rho_0
// dx/(2 eps0), E_N = -d_{N-1}/dx + rho_N dx/(2 eps0); periodic wrap uses
// S_{N-1}).  Everything up to the per-node values is integer, so the FP64
// work (slow on B300: 64-cycle latency, 2 lanes per clock per SM) is about
// twenty operations per node plus the global terms, done by one lane.  The
// cluster synchronises once: each CTA publishes integer moments of its slice
// (charge, sum of its local prefixes, sum of their running sums) and every
// CTA derives its offsets and the global terms from them in rank order.  The
// field-energy diagnostic is reduced in FP32.  V(t) advances by an exact
// rotation of each harmonic's (cos, sin) by 2 pi f dt per step.
// mode 0: field of the loaded state at t = 0; mode 1: end of a step
// (t = (step+1) dt, moments accumulated, counters advanced).
struct FieldPart {
    unsigned long long seg[2], all[2];  // interior / all-node raw charge of the slice
    u128 qp[2];                         // sum over slice m < N of the local prefix p_s[m]
    u128 qq[2];                         // sum over slice i < N of e_s[i] = sum_{c_lo <= m < i} p_s[m]
    unsigned long long r0[2];           // rank 0: raw deposit of node 0 (series-capacitor circuit)
};

template <int CL>
__device__ __forceinline__ void field_solve(const StepConst &P, int mode)
{
    namespace cg = cooperative_groups;
    cg::cluster_group cl = cg::this_cluster();
    unsigned long long *R_last = P.R_last;
    extern __shared__ __align__(16) double Ssh[];                    // [kFieldThreads + 1]: S at node c_lo - 1 + t
    __shared__ unsigned long long ured[kFieldThreads / 32][4];
    __shared__ u128 wred[kFieldThreads / 32][2];
    __shared__ float fred[kFieldThreads / 32];
    __shared__ FieldPart pub;                                       // this CTA's published moments
    __shared__ unsigned long long g_off[2], g_seg[2];               // slice prefix offset O_s, total interior charge
    __shared__ u128 g_qoff[2];                                      // Q_s[c_lo]
    __shared__ double g_b, g_d0, g_pm, g_phi0, g_qel;
    const int rank = (int)cl.block_rank();
    const int N = P.n_cells, nn = P.n_nodes, tid = threadIdx.x, ns = P.n_species;
    const int per_cta = (N + 1 + CL - 1) / CL;                      // <= kFieldThreads
    const int c_lo = min(rank * per_cta, N + 1), c_hi = min(c_lo + per_cta, N + 1);
    const int i = c_lo + tid;                                       // this thread's node
    const bool own = i < c_hi;
    Ctrl *ctrl = P.ctrl;
    const long long step = ctrl->step;
    const unsigned long long fe_n = ctrl->fe_n;
    const bool diag = mode == 1 && P.diag_interval > 0 && ((step + 1) % P.diag_interval) == 0;
    // the drive's phases, read now for the global terms of step 3 (thread 0 only)
    double drive_c[4] = {0.0, 0.0, 0.0, 0.0};
    if (tid == 0 && mode == 1 && !P.periodic)
        for (int h = 0; h < P.n_harm; ++h) drive_c[h] = ctrl->drive_c[h];

    // 1. raw deposit of the node (periodic: node N folds onto node 0); all loads issued first
    unsigned long long r[2] = {0ull, 0ull}, rs[2] = {0ull, 0ull}, rd[2] = {0ull, 0ull};
    double ps_old = 0.0;                                            // potential sum, read with the deposits
    const bool real = own && i < nn;
    if (real) {
        unsigned long long v[2][kDepositCopies];
#pragma unroll
        for (int s = 0; s < 2; ++s)
#pragma unroll
            for (int k = 0; k < kDepositCopies; ++k) v[s][k] = s < ns ? P.R[s][k * P.r_stride + i] : 0ull;
        if (mode == 1) {
            ps_old = P.phi_sum[i];
#pragma unroll
            for (int s = 0; s < 2; ++s)
                if (s < ns) {
                    rs[s] = P.Rsum[s * nn + i];
                    if (diag) rd[s] = P.Rdiag[s * nn + i];
                }
        }
#pragma unroll
        for (int s = 0; s < 2; ++s)
#pragma unroll
            for (int k = 0; k < kDepositCopies; ++k) r[s] += v[s][k];
        if (P.periodic && i == 0)
            for (int s = 0; s < ns; ++s)
                for (int k = 0; k < kDepositCopies; ++k) r[s] += P.R[s][k * P.r_stride + N];
        for (int s = 0; s < ns; ++s) {
            R_last[s * nn + i] = r[s];
            if (mode == 1) {
                P.Rsum[s * nn + i] = rs[s] + r[s];
                if (diag) P.Rdiag[s * nn + i] = rd[s] + r[s];
            }
        }
    }
    const bool interior = own && i >= 1 && i <= N - 1;
    // 2. local prefix p_s[i] (interior R from c_lo), its running sum e_s[i], slice moments
    unsigned long long pv[2], ptot[4];
    {
        const unsigned long long v4[4] = {interior ? r[0] : 0ull, interior ? r[1] : 0ull, real ? r[0] : 0ull,
                                          real ? r[1] : 0ull};
        unsigned long long ex4[4];
        block_exclusive_vec<unsigned long long, 4>(v4, ex4, ptot, ured);
        pv[0] = ex4[0] + v4[0];                                    // p_s[i] (inclusive)
        pv[1] = ex4[1] + v4[1];
    }
    u128 e[2], qp_tot[2], qq_tot[2];
    {
        const u128 v2[2] = {own && i < N ? (u128)pv[0] : (u128)0, own && i < N ? (u128)pv[1] : (u128)0};
        block_exclusive_vec<u128, 2>(v2, e, qp_tot, wred);          // e_s[i] = sum_{c_lo <= m < i} p_s[m]
        // the slice total of e_s[i] (a sum: no prefix needed)
        u128 w2[2] = {own && i < N ? e[0] : (u128)0, own && i < N ? e[1] : (u128)0};
        const int lane = tid & 31, warp = tid >> 5, nw = (int)(blockDim.x >> 5);
        for (int o = 16; o > 0; o >>= 1)
#pragma unroll
            for (int s = 0; s < 2; ++s) {
                const unsigned long long lo2 = __shfl_xor_sync(0xffffffffu, (unsigned long long)w2[s], o);
                const unsigned long long hi2 = __shfl_xor_sync(0xffffffffu, (unsigned long long)(w2[s] >> 64), o);
                w2[s] += ((u128)hi2 << 64) | lo2;
            }
        if (lane == 0) { wred[warp][0] = w2[0]; wred[warp][1] = w2[1]; }
        __syncthreads();
        qq_tot[0] = qq_tot[1] = (u128)0;
        if (tid == 0)
            for (int w = 0; w < nw; ++w) { qq_tot[0] += wred[w][0]; qq_tot[1] += wred[w][1]; }
    }
    if (tid == 0) {
        for (int s = 0; s < 2; ++s) {
            const bool sp = s < ns;
            pub.seg[s] = sp ? ptot[s] : 0ull;
            pub.all[s] = sp ? ptot[2 + s] : 0ull;
            pub.qp[s] = sp ? qp_tot[s] : (u128)0;
            pub.qq[s] = sp ? qq_tot[s] : (u128)0;
            pub.r0[s] = sp ? r[s] : 0ull;
        }
    }
    cl.sync();                                                      // the one exchange
    // 3. warp 0: lane r takes rank r's moments; integer offsets; lane 0 the FP64 globals
    if (tid < 32) {
        const int lane = tid;
        FieldPart q{};
        if (lane < CL) q = *cl.map_shared_rank(&pub, lane);
        const int r_lo = min(lane * per_cta, N + 1), r_hi = min(r_lo + per_cta, N + 1);
        const long long cnt = (lane < CL && min(r_hi, N) > r_lo) ? min(r_hi, N) - r_lo : 0;
        const u128 k1 = (u128)(cnt * (cnt - 1) / 2);                 // sum over slice i<N of (i - c_lo)
        unsigned long long off[2], segtot[2], alltot[2];
        u128 qoff[2], qn[2], sq[2];
        for (int s = 0; s < 2; ++s) {
            unsigned long long inc = q.seg[s], at = q.all[s];
            const u128 A0 = q.qp[s];
            for (int o = 1; o < CL; o <<= 1) {
                const unsigned long long y = __shfl_up_sync(0xffffffffu, inc, o);
                if (lane >= o) inc += y;
                at += __shfl_xor_sync(0xffffffffu, at, o);
            }
            off[s] = inc - q.seg[s];
            segtot[s] = __shfl_sync(0xffffffffu, inc, CL - 1);
            alltot[s] = __shfl_sync(0xffffffffu, at, 0);
            const u128 A = (u128)cnt * off[s] + A0;                 // sum of P_s[m] over the slice's m < N
            u128 ainc = A;
            for (int o = 1; o < CL; o <<= 1) {
                const u128 y = shfl_up_u128(ainc, o);
                if (lane >= o) ainc += y;
            }
            qoff[s] = ainc - A;                                     // Q_s[r_lo]
            qn[s] = shfl_u128(ainc, CL - 1);                        // Q_s[N]
            u128 B = (u128)cnt * qoff[s] + k1 * off[s] + q.qq[s];   // sum of Q_s[i] over the slice's i < N
            for (int o = 1; o < CL; o <<= 1) {
                const unsigned long long lo2 = __shfl_xor_sync(0xffffffffu, (unsigned long long)B, o);
                const unsigned long long hi2 = __shfl_xor_sync(0xffffffffu, (unsigned long long)(B >> 64), o);
                B += ((u128)hi2 << 64) | lo2;
            }
            sq[s] = shfl_u128(B, 0);                                // sum_{i<N} Q_s[i]
        }
        const unsigned long long my_off0 = __shfl_sync(0xffffffffu, off[0], rank);
        const unsigned long long my_off1 = __shfl_sync(0xffffffffu, off[1], rank);
        const u128 my_q0 = shfl_u128(qoff[0], rank), my_q1 = shfl_u128(qoff[1], rank);
        if (lane == 0) {
            double phi0 = 0.0;                                      // electrode voltage at this solve's time
            if (!P.periodic) {
                if (mode == 0) phi0 = P.v_init;
                else for (int h = 0; h < P.n_harm; ++h) phi0 = fma(P.harm_a[h], drive_c[h], phi0);
            }
            double b = P.bg_r;
            if (P.periodic) b = -(P.cq[0] * (double)(long long)alltot[0] + P.cq[1] * (double)(long long)alltot[1]) * P.inv_n;
            const double Nd = (double)N;
            const double TN = fma(P.cq[0], u128_to_double(qn[0]), fma(P.cq[1], u128_to_double(qn[1]), b * (0.5 * Nd * (Nd - 1.0))));
            double q_el = 0.0;
            if (P.circuit && mode == 1) {
                // (circuit 2: phi0 holds J(t^{n+1}) and c_blk = 0)
                // series capacitor: the electrode's charge takes this step's
                // absorbed and emitted particles; then phi_0 (C + eps0/L) =
                // Q + C V + (eps0/L) T_N + rho_0 dx/2, with (eps0/L) T_N the
                // (eps0/dx) phi_1 of the solution for phi_0 = 0
                double dq = P.qw[0] * (double)ctrl->st_abs0[0];
                if (ns > 1) dq += P.qw[1] * (double)ctrl->st_abs0[1];
                dq -= P.qw[0] * (double)ctrl->st_see0;
                if (P.circuit == 2) dq += P.dt * phi0;
                q_el = ctrl->q_el + dq;
                const double rho0_half =
                    fma(P.r0c[0], (double)(long long)q.r0[0], fma(P.r0c[1], (double)(long long)q.r0[1], P.bg_half));
                phi0 = (q_el + P.c_blk * phi0 + P.eps0_L * TN + rho0_half) * P.inv_cap_eps0_L;
            }
            const double d0 = (TN - phi0) * P.inv_n;
            double pm = 0.0;
            if (P.periodic) {                                       // mean of phi_0 + i d_0 - T_i over i < N
                const double sumT = fma(P.cq[0], u128_to_double(sq[0]),
                                        fma(P.cq[1], u128_to_double(sq[1]), b * (Nd * (Nd - 1.0) * (Nd - 2.0) / 6.0)));
                pm = (fma(d0, 0.5 * Nd * (Nd - 1.0), phi0 * Nd) - sumT) * P.inv_n;
            }
            g_off[0] = my_off0; g_off[1] = my_off1;
            g_qoff[0] = my_q0; g_qoff[1] = my_q1;
            g_seg[0] = segtot[0]; g_seg[1] = segtot[1];
            g_b = b; g_d0 = d0; g_pm = pm; g_phi0 = phi0; g_qel = q_el;
        }
    }
    cl.barrier_arrive();                                          // done reading the other slices
    __syncthreads();
    if (real)                                                     // every rank has read R
        for (int s = 0; s < ns; ++s)
            for (int k = 0; k < kDepositCopies; ++k) P.R[s][k * P.r_stride + i] = 0ull;
    if (own && i == N)
        for (int s = 0; s < ns; ++s)
            for (int k = 0; k < kDepositCopies; ++k) P.R[s][k * P.r_stride + N] = 0ull;
    const double b = g_b, d0 = g_d0, pm = g_pm, phi0 = g_phi0;
    const double cq0 = P.cq[0], cq1 = ns > 1 ? P.cq[1] : 0.0;
    // 4. S_i once per node (P_s[i] = O_s + p_s[i]); slot 0 holds S_{c_lo - 1} (P = O_s)
    if (own) {
        const double S = (i < N) ? fma(cq0, (double)(long long)(g_off[0] + pv[0]),
                                       fma(cq1, (double)(long long)(g_off[1] + pv[1]), b * (double)i))
                                 : 0.0;
        Ssh[tid + 1] = S;
    }
    if (tid == 0) {
        const int j = c_lo - 1;
        double S = 0.0;
        if (j >= 0) S = fma(cq0, (double)(long long)g_off[0], fma(cq1, (double)(long long)g_off[1], b * (double)j));
        else if (P.periodic)                                        // left of node 0 is node N-1
            S = fma(cq0, (double)(long long)g_seg[0], fma(cq1, (double)(long long)g_seg[1], b * (double)(N - 1)));
        Ssh[0] = S;
    }
    __syncthreads();
    // 5. node field, potential, FP32 copy for the gather, field energy (FP32), potential sum
    float fe = 0.0f;
    bool bad = false;
    if (real) {
        double E;
        if (!P.periodic && (i == 0 || i == N)) {
            double rq = P.bg_charge;                                // charge density of the wall node
            for (int s = 0; s < ns; ++s) rq = fma(P.rho_wall[s], (double)(long long)r[s], rq);
            E = i == 0 ? -d0 * P.inv_dx - rq * P.half_dx_eps0 : (Ssh[tid] - d0) * P.inv_dx + rq * P.half_dx_eps0;
            if (mode == 0 && P.circuit && i == 0) {                // at load the capacitor is uncharged
                ctrl->q_el = P.eps0 * E;
                ctrl->st_abs0[0] = ctrl->st_abs0[1] = 0ull;
                ctrl->st_see0 = 0ull;
            }
            fe = 0.5f * (float)E * (float)E;
        } else {
            E = (Ssh[tid + 1] + Ssh[tid] - 2.0 * d0) * P.inv_2dx;
            fe = (float)E * (float)E;
        }
        // Q_s[i] = Q_s[c_lo] + (i - c_lo) O_s + e_s[i]
        const unsigned long long k = (unsigned long long)tid;
        double T = b * (0.5 * (double)i * (double)(i - 1));
        T = fma(cq0, u128_to_double(g_qoff[0] + (u128)k * g_off[0] + e[0]), T);
        if (ns > 1) T = fma(cq1, u128_to_double(g_qoff[1] + (u128)k * g_off[1] + e[1]), T);
        double ph = fma((double)i, d0, phi0) - T - pm;
        if (!P.periodic && i == N) ph = 0.0;
        if (P.no_field) { E = 0.0; ph = 0.0; fe = 0.0f; }    // swarm: only the imposed field acts
        P.E[i] = E;
        P.phi[i] = ph;
        const float e32 = (float)E;                               // both cells that touch node i
        if (i < N) P.E32p[i].x = e32;
        if (i > 0) P.E32p[i - 1].y = e32;
        else if (P.periodic) P.E32p[N - 1].y = e32;
        if (mode == 1) P.phi_sum[i] = ps_old + ph;
        bad = !finite_bits(ph) || !finite_bits(E);
    }
    for (int o = 16; o > 0; o >>= 1) fe += __shfl_xor_sync(0xffffffffu, fe, o);
    if ((tid & 31) == 0) fred[tid >> 5] = fe;
    const bool any_bad = __syncthreads_or(bad);
    if (tid == 0) {
        float t = 0.0f;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += fred[w];
        if (any_bad) atomicOr(&ctrl->err, kErrNumeric);
        if (mode == 1) {                                          // kFieldCluster slots per entry
            double *fe_slot = P.fe_hist + (fe_n % (unsigned long long)P.fe_cap) * kFieldCluster;
            fe_slot[rank] = (double)t * P.fe_c;
            if (rank == 0)
                for (int r2 = CL; r2 < kFieldCluster; ++r2) fe_slot[r2] = 0.0;
        }
    }
    cl.barrier_wait();                                            // no CTA leaves while read remotely
    // Every rank has read the drive phases and counts (its global terms come
    // before its barrier arrival): rank 0 advances them for the next step.
    if (rank == 0 && tid == 0 && mode == 1) {
        ctrl->fe_n = fe_n + 1;
        ctrl->n_steps_acc += 1;
        if (diag) ctrl->n_diag_acc += 1;
        for (int s = 0; s < ns; ++s) {
            unsigned long long nt = ctrl->n_total[s];
            if (nt > P.cap[s]) nt = P.cap[s];
            ctrl->n_total[s] = nt;
            ctrl->n_active[s] = nt;
        }
        for (int h = 0; h < P.n_harm; ++h) {                      // advance each harmonic's phase by 2 pi f dt
            const double c = ctrl->drive_c[h], sn = ctrl->drive_s[h];
            ctrl->drive_c[h] = c * P.rot_c[h] - sn * P.rot_s[h];
            ctrl->drive_s[h] = sn * P.rot_c[h] + c * P.rot_s[h];
        }
        ctrl->step = step + 1;
        if (P.circuit) {
            ctrl->q_el = g_qel;
            ctrl->st_abs0[0] = ctrl->st_abs0[1] = 0ull;
            ctrl->st_see0 = 0ull;
        }
    }
}

// Waits for the step's particle kernels (programmatic launch), then lets the
// next step's electron kernel start its prologue on the other SMs.
__global__ void __cluster_dims__(kFieldCluster, 1, 1) __launch_bounds__(kFieldThreads)
    k_field(const __grid_constant__ StepConst P, int mode)
{
    grid_dep_wait();
    grid_dep_launch();
    field_solve<kFieldCluster>(P, mode);
}

// Smallest power-of-two cluster whose CTAs hold a grid's nodes one per thread.
__host__ __device__ constexpr int field_cluster_for(int n_cells)
{
    return n_cells + 1 <= kFieldThreads ? 1 : n_cells + 1 <= 2 * kFieldThreads ? 2 : n_cells + 1 <= 4 * kFieldThreads ? 4 : 8;
}

// Threads of a field CTA: one per node of its slice, in whole warps (the
// block scans and barriers cost in proportion to the warps).
__host__ __device__ constexpr int field_threads_for(int n_cells, int cl)
{
    return ((n_cells + 1 + cl - 1) / cl + 31) / 32 * 32 < 64 ? 64 : ((n_cells + 1 + cl - 1) / cl + 31) / 32 * 32;
}

// The batch's field solves, one launch per cluster size: cluster k solves case
// case_of[k] (the cases whose grids need CL CTAs).  The last launch of the
// step also resets the batch work-item counter for the next step.  Clusters
// of 4 and 8 CTAs run two CTAs an SM (56 registers, some spilled): at one an
// SM, with 96 registers, a sweep's largest grids solved in about four waves.
template <int CL>
__global__ void __cluster_dims__(CL, 1, 1) __launch_bounds__(kFieldThreads, CL >= 4 ? 2 : 1)
    k_batch_field(const StepConst *__restrict__ cases, const int *__restrict__ case_of, int mode, unsigned *next_item)
{
    field_solve<CL>(cases[case_of[blockIdx.x / CL]], mode);
    if (blockIdx.x == 0 && threadIdx.x == 0 && next_item) *next_item = 0u;
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

// Warp-aggregated increment of the shared counter cnt[c]: each run of
// consecutive lanes holding the same cell shares one atomic (sorted or nearly
// sorted particles would otherwise serialise 32 atomics on one address).  A
// cell that appears in several runs of the warp gets one reservation per run,
// so the ranks stay unique for any input.  Every lane of the warp calls it;
// lanes with `active` false take no part.  Returns the counter's old value plus
// the lane's rank within its run.
__device__ __forceinline__ unsigned warp_agg_inc(unsigned *cnt, int c, bool active)
{
    const int lane = threadIdx.x & 31;
    const int key = active ? c : -1;
    const int prev = __shfl_up_sync(0xffffffffu, key, 1);
    const unsigned starts = __ballot_sync(0xffffffffu, lane == 0 || key != prev);
    const int s0 = 31 - __clz(starts & (0xffffffffu >> (31 - lane)));      // this lane's run start
    const unsigned above = lane == 31 ? 0u : starts & (0xffffffffu << (lane + 1));
    const int e0 = above ? __ffs(above) - 1 : 32;                         // its end
    unsigned old = 0u;
    if (active && lane == s0) old = atomicAdd(&cnt[c], (unsigned)(e0 - s0));
    old = __shfl_sync(0xffffffffu, old, s0);
    return old + (unsigned)(lane - s0);
}

// Loops below advance whole warps together (blockDim a multiple of 32), so
// that every lane reaches the warp-wide calls, and issue kSortUnroll rounds
// of loads before they use them.
constexpr int kSortUnroll = 4;
// Sort key of a cell word: a case's particles (CLOCK) carry their collision
// clock above the cell bits; the stand-alone entry point takes plain cells.
template <bool CLOCK> __device__ __forceinline__ int sort_key(int w) { return (CLOCK && w >= 0) ? (w & kCellMask) : w; }

// Block `blk` of `nblk` counting one species' particles (a case's, or the
// stand-alone entry point's) into counts[cell].
template <bool CLOCK>
__device__ __forceinline__ void cells_count(SortHalves H, const int32_t *cur_dev, const unsigned long long *n_dev,
                                            long long n_host, int N, unsigned *counts, int blk, int nblk)
{
    extern __shared__ unsigned cnt_s[];
    for (int j = threadIdx.x; j < N; j += blockDim.x) cnt_s[j] = 0u;
    __syncthreads();
    const SpeciesBufs A = H.h[cur_dev ? *cur_dev : 0];
    const long long n = sort_count_of(n_dev, n_host);
    const int lane = threadIdx.x & 31;
    const long long stride = (long long)nblk * blockDim.x;
    for (long long w = blk * (long long)blockDim.x + (threadIdx.x & ~31); w < n; w += kSortUnroll * stride) {
        int cs[kSortUnroll];                            // loads first, then the counts
#pragma unroll
        for (int u = 0; u < kSortUnroll; ++u) {
            const long long i = w + u * stride + lane;
            cs[u] = i < n ? sort_key<CLOCK>(A.cell[i]) : -1;
        }
#pragma unroll
        for (int u = 0; u < kSortUnroll; ++u) warp_agg_inc(cnt_s, cs[u], cs[u] >= 0 && cs[u] < N);
    }
    __syncthreads();
    for (int j = threadIdx.x; j < N; j += blockDim.x)
        if (cnt_s[j]) atomicAdd(&counts[j], cnt_s[j]);
}

template <bool CLOCK>
__global__ void k_cells_count(SortHalves H, const int32_t *cur_dev, const unsigned long long *n_dev, long long n_host,
                              int N, unsigned *counts)
{
    cells_count<CLOCK>(H, cur_dev, n_dev, n_host, N, counts, blockIdx.x, gridDim.x);
}

// cursor[j] = sum_{k<j} counts[k]; cursor[N] = total (one CTA, exact: counts < 2^53)
__device__ __forceinline__ void cells_scan(const unsigned *counts, int N, unsigned long long *cursor)
{
    extern __shared__ __align__(16) double ssm[];
    __shared__ double red[32];
    for (int j = threadIdx.x; j < N; j += blockDim.x) ssm[j] = (double)counts[j];
    __syncthreads();
    block_scan_inclusive(ssm, N, red);
    for (int j = threadIdx.x; j < N; j += blockDim.x) cursor[j] = (unsigned long long)(ssm[j] - (double)counts[j]);
    if (threadIdx.x == 0) cursor[N] = (unsigned long long)ssm[N - 1];
}

__global__ void __launch_bounds__(1024) k_cells_scan(const unsigned *counts, int N, unsigned long long *cursor)
{
    cells_scan(counts, N, cursor);
}

// Exclusive prefix sums out[j] = sum_{k<j} in[j] of N shared counters by the
// whole CTA (each thread a run of consecutive counters); returns the total.
__device__ __forceinline__ unsigned block_exclusive_u32(const unsigned *in, unsigned *out, int N, unsigned *wsum)
{
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = (int)(blockDim.x >> 5);
    const int per = (N + (int)blockDim.x - 1) / (int)blockDim.x;
    const int j0 = tid * per;
    unsigned own = 0u;
    for (int k = 0; k < per; ++k)
        if (j0 + k < N) own += in[j0 + k];
    unsigned x = own;                                   // inclusive scan over the warp
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) wsum[warp] = x;
    __syncthreads();
    if (warp == 0) {
        unsigned w = lane < nw ? wsum[lane] : 0u;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        if (lane < nw) wsum[lane] = w;
    }
    __syncthreads();
    unsigned run = (warp > 0 ? wsum[warp - 1] : 0u) + x - own;
    for (int k = 0; k < per; ++k)
        if (j0 + k < N) { out[j0 + k] = run; run += in[j0 + k]; }
    return wsum[nw - 1];
}

// Scatter of the counting sort.  Each CTA takes one contiguous chunk of the
// particles (chunk = n / blocks, in whole warps) and moves it in tiles of
// kScatterTile, kScatterPer particles a thread, all loads first:
//   1. ranks within the tile's cells (shared counters, one atomic per run of
//      equal cells in a warp);
//   2. the cells' offsets in the tile (a prefix sum over the cells), and one
//      range per touched cell reserved on the global cursor;
//   3. the tile laid out in shared memory in cell order;
//   4. stores from the cell-ordered tile: consecutive threads write
//      consecutive slots of a cell's run, so that a run of k particles costs
//      about k/8 sectors an array instead of up to one sector a particle.
// Shared memory: scatter_smem(N).  The order within a cell is unspecified.
constexpr int kScatterThreads = 512;
constexpr int kScatterPer = 4;
constexpr int kScatterTile = kScatterThreads * kScatterPer;
constexpr int kScatterArrays = 7;                       // cell word, off, vx, vy, vz, id, z
__host__ __device__ constexpr size_t scatter_smem(int N)
{
    return (size_t)N * 16u + (size_t)kScatterTile * kScatterArrays * 4u;
}
template <bool CLOCK>
__device__ __forceinline__ void cells_scatter(SortHalves H, const int32_t *cur_dev, const unsigned long long *n_dev,
                                              long long n_host, int N, unsigned long long *cursor, int blk, int nblk)
{
    extern __shared__ __align__(16) unsigned char xsm[];
    unsigned long long *gbase = reinterpret_cast<unsigned long long *>(xsm);   // [N] reserved global slot
    unsigned *tcnt = reinterpret_cast<unsigned *>(xsm + 8 * (size_t)N);         // [N] tile count
    unsigned *toff = tcnt + N;                                                   // [N] tile offset
    uint32_t *stg = reinterpret_cast<uint32_t *>(xsm + 16 * (size_t)N);         // [arrays][kScatterTile]
    __shared__ unsigned wsum[kScatterThreads / 32];
    const int tid = threadIdx.x;
    for (int j = tid; j < N; j += kScatterThreads) tcnt[j] = 0u;
    const int half = cur_dev ? *cur_dev : 0;
    const SpeciesBufs A = H.h[half], D = H.h[half ^ 1];
    const long long n = sort_count_of(n_dev, n_host);
    long long chunk = (n + nblk - 1) / nblk;
    chunk = (chunk + 31) & ~31ll;
    const long long lo = min((long long)blk * chunk, n), hi = min(lo + chunk, n);
    const bool has_z = A.z != nullptr;
    __syncthreads();
    for (long long t0 = lo; t0 < hi; t0 += kScatterTile) {
        int key[kScatterPer];
        uint32_t val[kScatterPer][kScatterArrays];
#pragma unroll
        for (int u = 0; u < kScatterPer; ++u) {             // all loads first (coalesced)
            const long long i = t0 + (long long)u * kScatterThreads + tid;
            const bool in = i < hi;
            const int c = in ? A.cell[i] : -1;
            val[u][0] = (uint32_t)c;
            val[u][1] = in ? __float_as_uint(A.off[i]) : 0u;
            val[u][2] = in ? __float_as_uint(A.vx[i]) : 0u;
            val[u][3] = in ? __float_as_uint(A.vy[i]) : 0u;
            val[u][4] = in ? __float_as_uint(A.vz[i]) : 0u;
            val[u][5] = in ? A.id[i] : 0u;
            val[u][6] = (in && has_z) ? __float_as_uint(A.z[i]) : 0u;
            key[u] = sort_key<CLOCK>(c);
        }
        unsigned rk[kScatterPer];
#pragma unroll
        for (int u = 0; u < kScatterPer; ++u) rk[u] = warp_agg_inc(tcnt, key[u], key[u] >= 0 && key[u] < N);
        __syncthreads();
        const unsigned m = block_exclusive_u32(tcnt, toff, N, wsum);   // live particles of the tile
        for (int j = tid; j < N; j += kScatterThreads) {
            const unsigned k = tcnt[j];
            if (k) gbase[j] = atomicAdd(&cursor[j], (unsigned long long)k);
        }
        __syncthreads();
#pragma unroll
        for (int u = 0; u < kScatterPer; ++u) {
            if (key[u] < 0 || key[u] >= N) continue;
            const unsigned sl = toff[key[u]] + rk[u];
#pragma unroll
            for (int a = 0; a < kScatterArrays; ++a) stg[a * kScatterTile + sl] = val[u][a];
        }
        __syncthreads();
        for (unsigned j = tid; j < m; j += kScatterThreads) {
            const int c = (int)stg[j];
            const int k = sort_key<CLOCK>(c);
            const unsigned long long p = gbase[k] + (j - toff[k]);
            tcnt[k] = 0u;                                   // every touched cell has a particle here
            D.cell[p] = c;
            D.off[p] = __uint_as_float(stg[kScatterTile + j]);
            D.vx[p] = __uint_as_float(stg[2 * kScatterTile + j]);
            D.vy[p] = __uint_as_float(stg[3 * kScatterTile + j]);
            D.vz[p] = __uint_as_float(stg[4 * kScatterTile + j]);
            D.id[p] = stg[5 * kScatterTile + j];
            if (has_z) D.z[p] = __uint_as_float(stg[6 * kScatterTile + j]);
        }
        __syncthreads();                                    // the tile's reads before the next tile's writes
    }
}

template <bool CLOCK>
__global__ void __launch_bounds__(kScatterThreads, 1) k_cells_scatter(SortHalves H, const int32_t *cur_dev,
                                                          const unsigned long long *n_dev, long long n_host, int N,
                                                          unsigned long long *cursor)
{
    cells_scatter<CLOCK>(H, cur_dev, n_dev, n_host, N, cursor, blockIdx.x, gridDim.x);
}

// case epilogue: the sorted half becomes current; counts reset for next time
__device__ __forceinline__ void sort_finish(const StepConst &P, int sp, const unsigned long long *total, int blk,
                                            int nblk)
{
    const int N = P.n_cells;
    if (blk == 0 && threadIdx.x == 0) {
        Ctrl *ctrl = P.ctrl;
        const unsigned long long live = *total;
        ctrl->cur[sp] ^= 1;
        ctrl->n_total[sp] = live;
        ctrl->n_active[sp] = live;
        ctrl->n_dead[sp] = 0ull;
    }
    for (int j = blk * blockDim.x + threadIdx.x; j < N; j += nblk * blockDim.x) P.sort_count[j] = 0u;
}

__global__ void k_sort_finish(const __grid_constant__ StepConst P, int sp, const unsigned long long *total)
{
    sort_finish(P, sp, total, blockIdx.x, gridDim.x);
}

// The same sort for species sp of every case of a batch in one launch per
// kernel.  The count and scatter kernels take (case, block, blocks) items in
// case order, about one block per kSortItemParticles particles of the case,
// so that the few cases in flight at a time keep their scattered writes in L2
// until whole sectors are written; the scan and the epilogue take one block
// (scan) or a few (epilogue) per case.
struct SortItem {
    int case_idx, blk, nblk;
};
constexpr long long kSortItemParticles = 16384;
__device__ __forceinline__ SortHalves case_halves(const StepConst &P, int sp)
{
    return SortHalves{{P.buf[sp][0], P.buf[sp][1]}};
}
__global__ void k_batch_cells_count(const StepConst *__restrict__ cases, const SortItem *__restrict__ items, int sp)
{
    const SortItem it = items[blockIdx.x];
    const StepConst &P = cases[it.case_idx];
    if (sp >= P.n_species) return;
    cells_count<true>(case_halves(P, sp), &P.ctrl->cur[sp], &P.ctrl->n_active[sp], 0, P.n_cells, P.sort_count,
                      it.blk, it.nblk);
}
__global__ void __launch_bounds__(1024) k_batch_cells_scan(const StepConst *__restrict__ cases, int sp)
{
    const StepConst &P = cases[blockIdx.x];
    if (sp >= P.n_species) return;
    cells_scan(P.sort_count, P.n_cells, P.sort_cursor);
}
__global__ void __launch_bounds__(kScatterThreads, 1) k_batch_cells_scatter(const StepConst *__restrict__ cases,
                                                                const SortItem *__restrict__ items, int sp)
{
    const SortItem it = items[blockIdx.x];
    const StepConst &P = cases[it.case_idx];
    if (sp >= P.n_species) return;
    cells_scatter<true>(case_halves(P, sp), &P.ctrl->cur[sp], &P.ctrl->n_active[sp], 0, P.n_cells, P.sort_cursor,
                        it.blk, it.nblk);
}
__global__ void k_batch_sort_finish(const StepConst *__restrict__ cases, int sp)
{
    const StepConst &P = cases[blockIdx.y];
    if (sp >= P.n_species) return;
    sort_finish(P, sp, P.sort_cursor + P.n_cells, blockIdx.x, gridDim.x);
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
