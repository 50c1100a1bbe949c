"""Host logic of the autotuner's sort-interval choice (csrc/sort_interval.h),
compiled with the host C++ compiler and driven from here (no GPU)."""
import math
import os
import shutil
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2609_17151_b300", "csrc")

DRIVER = r"""
#include "sort_interval.h"
#include <cstdio>
#include <vector>
int main() {
    int n; double ts; int kmin, kmax;
    while (std::scanf("%d %lf %d %d", &n, &ts, &kmin, &kmax) == 4) {
        std::vector<double> t(n);
        for (auto &x : t) std::scanf("%lf", &x);
        const pic::SortIntervalFit f = pic::choose_sort_interval(t.data(), n, ts, kmin, kmax);
        std::printf("%d %.17g\n", f.K, f.slope);
    }
    return 0;
}
"""


@pytest.fixture(scope="module")
def chooser(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    d = tmp_path_factory.mktemp("sortk")
    src, exe = d / "drv.cpp", d / "drv"
    src.write_text(DRIVER)
    subprocess.check_call([cxx, "-O1", "-std=c++17", "-I", CSRC, str(src), "-o", str(exe)])

    def run(t, ts, kmin=4, kmax=1024):
        inp = f"{len(t)} {ts!r} {kmin} {kmax}\n" + " ".join(repr(float(x)) for x in t) + "\n"
        out = subprocess.run([str(exe)], input=inp, capture_output=True, text=True, check=True).stdout.split()
        return int(out[0]), float(out[1])
    return run


def brute_force(t, ts, slope, kmin=4, kmax=1024):
    """The same cost model written out: mean cost per step of a period K."""
    n = len(t)
    h = np.arange(n // 2, n)
    b, a = np.polyfit(h + 1.0, np.asarray(t)[h], 1)
    t_end = a + b * n
    best, kbest = None, None
    for K in range(kmin, kmax + 1):
        ext = [t[k - 1] if k <= n else t_end + slope * (k - n) for k in range(1, K + 1)]
        cost = (sum(ext) + ts) / K
        if best is None or cost < best:
            best, kbest = cost, K
    return kbest


def test_flat_step_times_never_shorten_the_period(chooser):
    K, slope = chooser([1.0] * 32, 10.0)
    assert K == 1024 and slope == 0.0


def test_linear_growth_gives_the_square_root_law(chooser):
    # t(k) = 1 + b k: mean cost 1 + b (K+1)/2 + ts/K, minimised near sqrt(2 ts / b)
    b, ts = 0.01, 5.0
    t = [1.0 + b * k for k in range(1, 33)]
    K, slope = chooser(t, ts)
    assert slope == pytest.approx(b, rel=1e-9)
    assert abs(K - math.sqrt(2 * ts / b)) <= 1.0


def test_saturating_loss_of_order_with_a_costly_sort_keeps_a_long_period(chooser):
    t = [1.0 + 0.5 * (1 - math.exp(-k / 3.0)) for k in range(1, 33)]
    K, slope = chooser(t, 20.0)
    assert K >= 512                     # the tail's small residual growth still counts, noise-free
    assert slope < 1e-3
    assert K == brute_force(t, 20.0, slope)


def test_saturating_loss_of_order_with_a_cheap_sort_sorts_often(chooser):
    t = [1.0 + 0.5 * (1 - math.exp(-k / 3.0)) for k in range(1, 33)]
    K, _ = chooser(t, 0.3)
    assert 4 <= K < 16
    assert K == brute_force(t, 0.3, 0.0)


def test_timing_noise_alone_does_not_shorten_the_period(chooser):
    rng = np.random.default_rng(7)
    for trial in range(20):
        t = 1.0 + 0.01 * rng.standard_normal(32)
        K, _ = chooser(list(t), 1.0)
        assert K >= 256, (trial, K)


def test_accumulating_dead_slots_bound_the_period(chooser):
    # a transient, then growth that continues (absorbed slots): a finite period,
    # equal to the minimum of the model computed independently
    t = [1.0 + 0.3 * (1 - math.exp(-k / 2.0)) + 0.002 * k for k in range(1, 33)]
    K, slope = chooser(t, 2.0)
    assert 4 <= K < 1024
    assert slope > 0.0
    assert K == brute_force(t, 2.0, slope)


NORM_DRIVER = r"""
#include "sort_interval.h"
#include <cstdio>
#include <vector>
int main() {
    int n; double a0, a1, ts;
    while (std::scanf("%d %lf %lf %lf", &n, &a0, &a1, &ts) == 4) {
        std::vector<double> t(n);
        for (auto &x : t) std::scanf("%lf", &x);
        pic::normalise_to_count(t.data(), n, a0, a1);
        const pic::SortIntervalFit f = pic::choose_sort_interval(t.data(), n, ts, 4, 1024);
        std::printf("%d", f.K);
        for (double x : t) std::printf(" %.17g", x);
        std::printf("\n");
    }
    return 0;
}
"""


@pytest.fixture(scope="module")
def normaliser(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    d = tmp_path_factory.mktemp("sortnorm")
    src, exe = d / "drv.cpp", d / "drv"
    src.write_text(NORM_DRIVER)
    subprocess.check_call([cxx, "-O1", "-std=c++17", "-I", CSRC, str(src), "-o", str(exe)])

    def run(t, a0, a1, ts):
        line = f"{len(t)} {a0!r} {a1!r} {ts!r} " + " ".join(repr(float(x)) for x in t) + "\n"
        out = subprocess.run([str(exe)], input=line, capture_output=True, text=True, check=True).stdout.split()
        return int(out[0]), np.array([float(x) for x in out[1:]])
    return run


def test_growth_of_the_particle_count_is_not_taken_for_lost_order(normaliser):
    """Step times that grow only because the discharge gains particles (time
    per particle constant) rescale to a flat window, so the sort interval goes
    to its maximum; without a count change the times are left as they are,
    and growth beyond the count's still shortens the interval."""
    n = 32
    a0, a1 = 1.0e8, 1.1e8
    a = a0 + (a1 - a0) * (np.arange(n) + 0.5) / n
    t = 2.5 * a / a0                                         # ms, proportional to the count
    K, tn = normaliser(t, a0, a1, 8.0)
    assert np.allclose(tn, 2.5, rtol=1e-12) and K == 1024
    K0, t0 = normaliser(t, a0, a0, 8.0)
    assert np.array_equal(t0, t) and K0 < 200                # read as lost order: sorts often
    Kd, _ = normaliser(t * (1 + 0.004 * np.arange(n)), a0, a1, 8.0)
    assert Kd < 1024
