// sort_interval.h -- the autotuner's choice of the sort interval (host code).
//
// Right after a counting sort the step-kernel time t(k) of the k-th step
// grows as particles lose their cell order (which saturates) and as absorbed
// slots accumulate (which does not); a sort costs t_sort.  Given t(1..n)
// measured after one sort, t(k) beyond the window is extended linearly from
// the window's end with the slope fitted by least squares over the second
// half of the window, less two standard errors of that fit and not below
// zero (timing noise alone then leaves the period at its maximum).  The
// interval is the K in [k_min, k_max] that minimises the mean cost per step
// of a sort period, (sum_{k<=K} t(k) + t_sort) / K.
#pragma once
#include <algorithm>
#include <cmath>

namespace pic {

struct SortIntervalFit {
    int K;            // chosen interval
    double slope;     // growth per step used beyond the window (>= 0)
};

// Step times measured while the live particle count went from a0 to a1
// (taken as linear over the window), rescaled to the count at the window's
// start: a discharge that ionizes or loses particles changes the step time
// by itself, and only the growth that a sort removes (lost cell order,
// absorbed slots) belongs in the fit.
inline void normalise_to_count(double *t, int n, double a0, double a1)
{
    if (!(a0 > 0) || !(a1 > 0)) return;
    for (int k = 0; k < n; ++k) {
        const double a = a0 + (a1 - a0) * (k + 0.5) / n;
        t[k] *= a0 / a;
    }
}

inline SortIntervalFit choose_sort_interval(const double *t, int n, double t_sort, int k_min, int k_max)
{
    const int h0 = n / 2;
    const double m = n - h0;
    double hx = 0, hy = 0, hxx = 0, hxy = 0;
    for (int k = h0; k < n; ++k) {
        const double x = k + 1;
        hx += x; hy += t[k]; hxx += x * x; hxy += x * t[k];
    }
    const double b = (m * hxy - hx * hy) / (m * hxx - hx * hx);
    const double a = (hy - b * hx) / m;
    double ss = 0;                                       // residual sum of squares
    for (int k = h0; k < n; ++k) {
        const double d = t[k] - a - b * (k + 1);
        ss += d * d;
    }
    const double se = m > 2 ? std::sqrt(ss / (m - 2) / (hxx - hx * hx / m)) : 0.0;
    const double b_sig = std::max(0.0, b - 2.0 * se);
    const double t_end = a + b * n;
    SortIntervalFit f{k_max, b_sig};
    double sum = 0, best = 0;
    for (int K = 1; K <= k_max; ++K) {
        sum += K <= n ? t[K - 1] : t_end + b_sig * (K - n);
        const double cost = (sum + t_sort) / K;
        if (K >= k_min && (K == k_min || cost < best)) { best = cost; f.K = K; }
    }
    return f;
}

} // namespace pic
