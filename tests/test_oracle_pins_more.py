"""More pins of the FP64 oracle, for the parts a GPU-against-oracle comparison
cannot check by itself: ion-neutral collisions (paper §1's null-collision
method with ions scattering on the gas, §3.3's argon discharges), the Adam
update of the warm-start network, the EEPF binning (§3.2), the J.E power sum
and the Gauss field at an electrode node.  Each pin is fixed by mathematics
or by physics independent of the oracle's code, and names the mistake it
would catch."""
import math

import numpy as np
from scipy import stats

import oracle
from oracle import mlp as omlp
from paper_2609_17151_b300 import workloads as W

E = W.E_CHARGE
EPS0 = W.EPS0
KB = W.K_B
AMU = 1.66053906660e-27
M_XE = 131.293 * AMU


def _ion_case(n_cells=16, *, ion_mass, gas_mass, gas_temp, ng, kinds, dt, seed=5):
    """Field-free periodic box (swarm mode): no electrons, ions of `ion_mass`
    colliding with a gas of `gas_mass` through the synthetic Ar+ forms of
    `kinds` (ISO and/or CX)."""
    tabs = [t for t in W.argon_tables() if t["species"] == 1 and t["kind"] in kinds]
    cfg = dict(periodic=1, n_cells=n_cells, length=n_cells * 1e-4, dt=dt, gas_density=ng, gas_temp=gas_temp,
               gas_mass=gas_mass, species=[dict(q=-E, m=W.M_E, w=1e-6), dict(q=E, m=ion_mass, w=1e-6)],
               seed=seed, rewind=0, no_field=1, xsec=tabs)
    return cfg, tabs


def _analytic_numax(tabs, ng, mu):
    """max over the table grid of sum_k N sigma_k(eps) g(eps), g = sqrt(2 e eps / mu)"""
    e = W.table_energies()
    g = np.sqrt(2 * e * E / mu)
    return float(np.max(sum(ng * t["sigma"] * g for t in tabs)))


def _load_ions(c, v):
    n = v.shape[0]
    xi = np.random.default_rng(1).uniform(0, c.n_cells, n)
    c.load_particles(0, np.zeros(0), np.zeros(0), np.zeros(0), np.zeros(0), np.zeros(0, np.uint32))
    c.load_particles(1, xi, v[:, 0], v[:, 1], v[:, 2], np.arange(n, dtype=np.uint32))


def test_ion_numax_is_built_over_the_relative_speed_with_the_reduced_mass():
    """nu_max of the ions is the largest N sum_k sigma_k(eps) g over the grid,
    with g the relative speed at centre-of-mass energy eps (reduced mass mu):
    building it over the ion's own lab speed (mass m instead of mu) changes it
    by sqrt(m/mu)."""
    ng = 1e22
    for mi, mg in ((W.M_AR, W.M_AR), (M_XE, W.M_AR), (W.M_AR, M_XE)):
        cfg, tabs = _ion_case(ion_mass=mi, gas_mass=mg, gas_temp=300.0, ng=ng, kinds=(W.ISO, W.CX), dt=1e-9)
        c = oracle.Case(cfg)
        mu = mi * mg / (mi + mg)
        assert abs(c.numax(1) / _analytic_numax(tabs, ng, mu) - 1) < 1e-12


def test_ions_equilibrate_to_the_gas_temperature_for_unequal_masses():
    """Hot ions (10 T_g) scattering isotropically in the centre-of-mass frame
    on a Maxwellian gas relax to <m v^2/2> = (3/2) k T_g whatever the mass
    ratio (detailed balance of elastic collisions).  A wrong centre-of-mass
    velocity or swapped mass fractions m/(m+M), M/(m+M) would settle at
    another temperature when m != M (here Xe+ in Ar and Ar+ in Xe)."""
    tg = 300.0
    for mi, mg in ((M_XE, W.M_AR), (W.M_AR, M_XE)):
        mu = mi * mg / (mi + mg)
        ng = 1e24
        cfg, tabs = _ion_case(ion_mass=mi, gas_mass=mg, gas_temp=tg, ng=ng, kinds=(W.ISO,), dt=1.0)
        cfg["dt"] = 0.15 / _analytic_numax(tabs, ng, mu)
        c = oracle.Case(cfg)
        n = 8000
        rng = np.random.default_rng(11)
        v = rng.normal(0.0, math.sqrt(KB * 10 * tg / mi), (n, 3))
        _load_ions(c, v)
        c.step(400)
        ke = []
        for _ in range(40):
            c.step(10)
            p = c.particles(1)
            ke.append(np.mean(0.5 * mi * (p["vx"] ** 2 + p["vy"] ** 2 + p["vz"] ** 2)))
        ratio = float(np.mean(ke)) / (1.5 * KB * tg)
        assert abs(ratio - 1) < 0.03, (mi / mg, ratio)
        assert c.counters()["collisions"][1][0] > 20 * n            # many collisions per ion


def test_monoenergetic_ion_beam_process_counts_are_binomial():
    """Ar+ at a fixed speed through cold Ar (partner nearly at rest): per-process
    counts of one step follow Binomial(N, (1 - exp(-numax dt)) nu_k / numax),
    nu_k = N sigma_k(eps_cm) g computed here from the analytic forms at
    eps_cm = mu g^2 / (2e)."""
    e_grid = W.table_energies()
    eps_cm = float(e_grid[730])                 # ~ 24 eV
    mi = mg = W.M_AR
    mu = 0.5 * mi
    g = math.sqrt(2 * eps_cm * E / mu)
    ng = 3e21
    cfg, tabs = _ion_case(ion_mass=mi, gas_mass=mg, gas_temp=1e-3, ng=ng, kinds=(W.ISO, W.CX), dt=1.0)
    numax = _analytic_numax(tabs, ng, mu)
    cfg["dt"] = 0.7 / numax
    c = oracle.Case(cfg)
    n = 400_000
    v = np.zeros((n, 3))
    v[:, 0] = g
    _load_ions(c, v)
    c.step(1)
    cnt = c.counters()
    pnull = 1 - math.exp(-numax * cfg["dt"])
    for k, t in enumerate(tabs):
        p = pnull * ng * t["sigma"][730] * g / numax
        o = cnt["collisions"][1][k]
        mean, sd = n * p, math.sqrt(n * p * (1 - p))
        assert abs(o - mean) < 5 * sd, (t["kind"], o, mean, sd)
    assert abs(cnt["candidates"][1] - n * pnull) < 5 * math.sqrt(n * pnull * (1 - pnull))


def test_charge_exchange_leaves_the_ions_with_the_gas_maxwellian():
    """After charge exchange an ion carries its gas partner's velocity: a
    beam of Ar+ that has undergone charge exchange has the gas Maxwellian,
    each component normal with deviation sqrt(k T_g / M) and no memory of
    the beam."""
    mi = mg = W.M_AR
    tg = 300.0
    ng = 3e21
    cfg, tabs = _ion_case(ion_mass=mi, gas_mass=mg, gas_temp=tg, ng=ng, kinds=(W.CX,), dt=1.0)
    cfg["dt"] = 2.3 / _analytic_numax(tabs, ng, 0.5 * mi)      # P_null = 0.9
    c = oracle.Case(cfg)
    n = 20_000
    v = np.zeros((n, 3))
    v[:, 0] = math.sqrt(2 * 5.0 * E / (0.5 * mi))
    _load_ions(c, v)
    c.step(150)
    p = c.particles(1)
    vt = math.sqrt(KB * tg / mg)
    for comp in ("vx", "vy", "vz"):
        assert stats.kstest(p[comp] / vt, "norm").pvalue > 1e-4, comp
    assert abs(np.mean(p["vx"])) < 5 * vt / math.sqrt(n)


# --------------------------------------------------------------------------- Adam
def test_adam_first_steps_have_their_closed_forms():
    """Adam (Kingma & Ba, bias-corrected): the first step moves each parameter
    by -lr g/(|g| + eps); a second step with the same gradient moves it by the
    same amount; a second step with the opposite gradient moves it back by
    lr (1 - b1)/(1 + b1) g/|g|.  A wrong bias correction (b^(t-1), or none)
    or a swapped moment fails one of these."""
    rng = np.random.default_rng(2)
    g = rng.normal(0, 1, 1000) * rng.choice([1e-4, 1.0, 1e3], 1000)
    p0 = rng.normal(0, 0.1, 1000)
    lr, b1, b2, eps = 1e-3, 0.9, 0.999, 1e-8
    z = np.zeros_like(p0)
    p1, m1, v1 = omlp.adam(p0, g, z, z, 1, lr)
    step1 = lr * g / (np.abs(g) + eps)
    assert np.allclose(p0 - p1, step1, rtol=1e-9, atol=1e-15)
    p2, _, _ = omlp.adam(p1, g, m1, v1, 2, lr)
    assert np.allclose(p1 - p2, step1, rtol=1e-9, atol=1e-15)
    p2b, _, _ = omlp.adam(p1, -g, m1, v1, 2, lr)
    # m2 = -(1-b1)^2 g, mhat = -(1-b1)/(1+b1) g; v2 = (1-b2)(1+b2) g^2, vhat = g^2
    back = lr * (1 - b1) / (1 + b1) * g / (np.abs(g) + eps)
    assert np.allclose(p2b - p1, back, rtol=1e-6, atol=1e-15)


# --------------------------------------------------------------------------- EEPF
def test_eepf_of_a_maxwellian_follows_the_gamma_three_halves_law():
    """Electrons loaded Maxwellian at T: the energy of each is Gamma(3/2, T)
    distributed, so the EEPF counts of the central 10 % of the gap (0.25 eV
    bins, paper §3.2) match n_in (F(b+1) - F(b)) by a chi-square test.  A
    wrong bin width, a missing 1/2 in the energy or the wrong region fails."""
    T = 5.0
    n, N = 2_000_000, 64
    cfg = dict(periodic=1, n_cells=N, length=N * 1e-4, dt=1e-14, species=[dict(q=-E, m=W.M_E, w=1e-6)],
               seed=3, rewind=0, no_field=1, diag_interval=1)
    rng = np.random.default_rng(9)
    v = rng.normal(0, math.sqrt(T * E / W.M_E), (n, 3))
    xi = rng.uniform(0, N, n)
    c = oracle.Case(cfg)
    c.load_particles(0, xi, v[:, 0], v[:, 1], v[:, 2], np.arange(n, dtype=np.uint32))
    c.step(1)
    eepf = c.moments()["eepf"]
    p = c.particles(0)
    n_in = int(np.sum((p["xi"] >= 0.45 * N) & (p["xi"] < 0.55 * N)))
    edges = 0.25 * np.arange(241)
    prob = np.diff(stats.gamma.cdf(edges, a=1.5, scale=T))
    expected = n_in * prob
    ok = expected >= 5
    chi2 = float(np.sum((eepf[ok] - expected[ok]) ** 2 / expected[ok]))
    assert stats.chi2.sf(chi2, int(ok.sum()) - 1) > 1e-4, chi2
    assert abs(eepf.sum() - n_in * prob.sum()) < 5 * math.sqrt(n_in) + 1
    mean = float(np.sum(0.25 * (np.arange(240) + 0.5) * eepf) / eepf.sum())
    assert abs(mean / (1.5 * T) - 1) < 0.005, mean          # <eps> = 3T/2 (sd of the ratio ~ 0.2 %)


# --------------------------------------------------------------------------- J.E
def test_power_sum_satisfies_the_leapfrog_energy_identity():
    """For B = 0 the push is v^{n+1/2} - v^{n-1/2} = (q/m) (E_m + E_x) dt, with
    E_m = E^n(x^n) the mesh field and E_x the imposed one, so each step's
    mesh power sum J.E = sum q w v_x^{n+1/2} E_m obeys exactly (to FP64
    rounding) J.E dt = KE^{n+1/2} - KE^{n-1/2} - q w E_x dt sum (v^{n+1/2} +
    v^{n-1/2})_x / 2 + (q^2 w dt^2 / 2m) sum E_m (E_m + E_x).  A wrong sign or
    weight, a velocity at the wrong time level, or the imposed field counted
    in it fails."""
    cfg, parts = W.langmuir_case(seed=4, amp=0.05)
    cfg["diag_interval"] = 1
    cfg["E_ext"] = (30.0, 0.0, 0.0)           # excluded from the mesh power by definition
    c = oracle.Case(cfg)
    c.load_particles(0, W.as_xi(parts[0]), parts[0]["vx"], parts[0]["vy"], parts[0]["vz"], parts[0]["id"])
    c.step(0)
    sp = cfg["species"][0]
    q, m, w, dt, N = sp["q"], sp["m"], sp["w"], cfg["dt"], cfg["n_cells"]
    seen = 0.0
    for _ in range(12):
        before = c.particles(0)
        E_mesh = c.field()[1]
        c.reset_moments()
        c.step(1)
        after = c.particles(0)
        mo = c.moments()
        ib, ia = np.argsort(before["id"]), np.argsort(after["id"])
        vb = np.stack([before[k][ib] for k in ("vx", "vy", "vz")], 1)
        va = np.stack([after[k][ia] for k in ("vx", "vy", "vz")], 1)
        ke_b = 0.5 * m * w * np.sum(vb ** 2)
        ke_a = 0.5 * m * w * np.sum(va ** 2)
        xi = before["xi"][ib]
        j = np.floor(xi).astype(int)
        t = xi - j
        Ep = (1 - t) * E_mesh[j] + t * E_mesh[(j + 1) % N]
        Ex = cfg["E_ext"][0]
        rhs = ((ke_a - ke_b) - q * w * Ex * dt * 0.5 * np.sum(va[:, 0] + vb[:, 0])
               + q * q * w * dt * dt / (2 * m) * np.sum(Ep * (Ep + Ex)))
        lhs = mo["pw_sum"][0] * dt
        assert abs(lhs - rhs) <= 1e-9 * ke_a, (lhs, rhs)
        assert abs(mo["ke_sum"][0] - ke_a) <= 1e-12 * ke_a
        seen = max(seen, abs(lhs))
    assert seen > 1e-5 * ke_a                    # the identity is not trivially 0 = 0


# --------------------------------------------------------------------------- Gauss at an electrode
def test_uniform_charge_between_grounded_plates_gives_the_exact_field_at_every_node():
    """A uniform charge rho between grounded electrodes: phi = rho x (L - x) /
    (2 eps0) and E = -rho (L - 2x) / (2 eps0).  Second-order differences are
    exact on a parabola, and so is the electrode node's Gauss half-cell field
    E_0 = -(phi_1 - phi_0)/dx - rho_0 dx/(2 eps0); dropping the half-cell term
    leaves E_0 off by rho dx/(2 eps0)."""
    rho, N, L = 3e-4, 40, 2e-3
    cfg = dict(periodic=0, n_cells=N, length=L, dt=1e-12, bg_charge=rho,
               species=[dict(q=-E, m=W.M_E, w=1e-6)], seed=1, rewind=0)
    c = oracle.Case(cfg)
    c.load_particles(0, np.zeros(0), np.zeros(0), np.zeros(0), np.zeros(0), np.zeros(0, np.uint32))
    c.step(0)
    phi, Ef = c.field()
    x = np.arange(N + 1) * (L / N)
    scale = rho * L / (2 * EPS0)
    assert np.abs(phi - rho * x * (L - x) / (2 * EPS0)).max() <= 1e-12 * scale * L
    assert np.abs(Ef + rho * (L - 2 * x) / (2 * EPS0)).max() <= 1e-12 * scale
    assert abs(Ef[0] + scale) <= 1e-12 * scale and abs(Ef[-1] - scale) <= 1e-12 * scale


# --------------------------------------------------------------------------- collision clock
def _uniforms(n, seed):
    """23-bit uniforms ((r >> 9) + 1/2) 2^-23, exact in FP32, as the method draws them"""
    r = np.random.default_rng(seed).integers(0, 2**32, n, dtype=np.uint64)
    return (((r >> 9).astype(np.float64) + 0.5) * 2.0**-23).astype(np.float32)


def test_fp32_log_of_the_collision_clock_is_within_a_few_ulp():
    """-ln(u) of the clock (FP32 atanh series, Abramowitz and Stegun 4.1.27)
    against the FP64 logarithm: relative error below 3e-7 (a few FP32 ulp) at
    random and at extreme uniforms; a wrong series coefficient, range
    reduction or ln 2 fails."""
    u = np.concatenate([_uniforms(100_000, 1), np.float32([2.0**-24, 0.5, 1 - 2.0**-24, 0.70710677, 0.70710683,
                                                            0.25, 0.99, 1e-6])])
    got = np.array([oracle.neg_log_u32(float(x)) for x in u])
    want = -np.log(u.astype(np.float64))
    assert np.max(np.abs(got - want) / want) < 3e-7


def test_clock_gaps_follow_the_geometric_law():
    """The gap G = floor(-ln u / lam) of the clock has P(G = g) = e^{-g lam}
    (1 - e^{-lam}) (the number of non-candidate steps of the null-collision
    method, paper §4); gaps above 131071 steps are cut, with probability
    e^{-131072 lam}, into a continuation."""
    u = _uniforms(200_000, 2)
    lam = 0.05
    st = np.array([oracle.clock_state(float(x), lam) for x in u])
    assert np.all(st % 2 == 0)
    g = st // 2
    k = np.arange(80)
    p = np.exp(-k * lam) * (1 - np.exp(-lam))
    obs = np.bincount(np.minimum(g, 80), minlength=81)
    exp_ = np.append(p, np.exp(-80 * lam)) * u.size
    chi2 = float(np.sum((obs - exp_) ** 2 / exp_))
    assert stats.chi2.sf(chi2, 80) > 1e-4, chi2
    lam = 8e-6
    st = np.array([oracle.clock_state(float(x), lam) for x in u[:50_000]])
    cont = st % 2 == 1
    pc = math.exp(-131072 * lam)
    assert abs(cont.mean() - pc) < 5 * math.sqrt(pc * (1 - pc) / cont.size)
    assert np.all(st[cont] == 2 * oracle.CLOCK_MAX + 1) and np.all(st[~cont] // 2 <= oracle.CLOCK_MAX)
