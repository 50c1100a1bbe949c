"""Seeded synthetic workloads: case parameters, cross-section tables, particle loads.

This module only builds INPUTS (numbers a user would type into the case dialog
of the paper's §1, and initial particle states); it contains none of the
method's arithmetic.  The CUDA library and the CPU oracle both consume what it
returns, so that both start from identical states.

Every particle state is returned as a dict per species with
``cell`` (int32), ``off`` (float32, in [0, 1)), ``vx, vy, vz`` (float32, m/s)
and ``id`` (uint32); ``xi = cell + off`` is exact in FP64.
"""
from __future__ import annotations

import math

import numpy as np
from scipy.special import ndtri

# physical constants (CODATA 2018) used to build the inputs
E_CHARGE = 1.602176634e-19
M_E = 9.1093837015e-31
AMU = 1.66053906660e-27
K_B = 1.380649e-23
EPS0 = 8.8541878128e-12
TORR = 133.322368

M_AR = 39.948 * AMU
M_XE = 131.293 * AMU

ELASTIC, EXCITATION, IONIZATION, ISO, CX = 0, 1, 2, 3, 4


# --------------------------------------------------------------------------- tables
def table_energies(n: int = 1000, emin: float = 1e-3, emax: float = 1e3) -> np.ndarray:
    """Energies (eV) at which the synthetic tables are written: n log-spaced points."""
    return emin * np.exp(np.arange(n) * (math.log(emax / emin) / (n - 1)))


def argon_tables() -> list[dict]:
    """Synthetic analytic argon cross sections (m^2 vs eV) standing in for the
    LXCat data the paper uses: electron elastic (Ramsauer-like dip), one
    excitation at 11.5 eV and ionization at 15.8 eV; Ar+ on Ar isotropic
    elastic and charge exchange against the centre-of-mass energy."""
    e = table_energies()
    el = 1e-20 + 1.4e-19 * e**2 / (e**2 + 1.0) * np.exp(-e / 50.0)
    x = e / 11.5
    exc = np.where(e >= 11.5, 2.5e-20 * np.log(np.maximum(x, 1.0)) / x, 0.0)
    y = e / 15.8
    iz = np.where(e >= 15.8, 8e-20 * np.log(np.maximum(y, 1.0)) / y, 0.0)
    iso = 1.5e-19 / np.sqrt(1.0 + e)
    cx = 3e-19 * (1.0 + e) ** -0.1
    return [
        dict(species=0, kind=ELASTIC, threshold=0.0, energy=e, sigma=el),
        dict(species=0, kind=EXCITATION, threshold=11.5, energy=e, sigma=exc),
        dict(species=0, kind=IONIZATION, threshold=15.8, energy=e, sigma=iz),
        dict(species=1, kind=ISO, threshold=0.0, energy=e, sigma=iso),
        dict(species=1, kind=CX, threshold=0.0, energy=e, sigma=cx),
    ]


# --------------------------------------------------------------------------- loaders
def _split(xi: np.ndarray, n_cells: int):
    """cell/offset of positions in cell units, offset rounded to FP32 below 1."""
    cell = np.floor(xi).astype(np.int64)
    off = (xi - cell).astype(np.float32)
    one = off >= np.float32(1.0)
    off[one] = np.float32(0.0)
    cell[one] += 1
    cell %= n_cells
    return cell.astype(np.int32), off


def maxwellian_load(rng: np.random.Generator, n: int, n_cells: int, temp_ev: float, mass: float,
                    drift=(0.0, 0.0, 0.0), id_base: int = 0, lo: float = 0.0, hi: float | None = None) -> dict:
    """n particles uniform in [lo, hi) cells with a (drifting) Maxwellian at temp_ev."""
    hi = n_cells if hi is None else hi
    xi = rng.uniform(lo, hi, n)
    cell, off = _split(xi, n_cells)
    vt = math.sqrt(temp_ev * E_CHARGE / mass)
    v = rng.standard_normal((3, n)) * vt + np.asarray(drift, dtype=np.float64)[:, None]
    return dict(cell=cell, off=off, vx=v[0].astype(np.float32), vy=v[1].astype(np.float32),
                vz=v[2].astype(np.float32), id=(id_base + np.arange(n)).astype(np.uint32))


def as_xi(s: dict) -> np.ndarray:
    return s["cell"].astype(np.float64) + s["off"].astype(np.float64)


# --------------------------------------------------------------------------- cases
def langmuir_case(seed: int = 1, k_lambda_d: float = 0.4, n_cells: int = 64, ppc: int = 100,
                  amp: float = 0.01, n0: float = 2e14, te_ev: float = 3.0, wpdt: float = 0.1,
                  slab: int = 8):
    """Langmuir wave on an immobile ion background (paper §3.1: 2e14 m^-3, 3 eV,
    periodic, no gas), one wavelength in the box, then displaced by
    -(amp/k) sin(kx) so that dn/n = amp cos(kx).

    Quiet start: the N Maxwellian v_x quantiles are cut into slabs of `slab`
    neighbours; the particles of one slab sit on a uniform lattice of `slab`
    points spread over the whole box, so the density of modes 1..slab-1 stays
    near zero under free streaming while every velocity stays distinct (no
    cold beams).  The seed permutes the slab base positions and draws the
    (dynamically inert) v_y, v_z."""
    lam_d = math.sqrt(EPS0 * te_ev / (n0 * E_CHARGE))
    wp = math.sqrt(n0 * E_CHARGE**2 / (EPS0 * M_E))
    L = 2 * math.pi * lam_d / k_lambda_d
    k = 2 * math.pi / L
    N = n_cells * ppc
    assert N % slab == 0
    n_slab = N // slab
    dx = L / n_cells
    rng = np.random.default_rng(seed)
    vt = math.sqrt(te_ev * E_CHARGE / M_E)
    vx = vt * ndtri((np.arange(N) + 0.5) / N)
    base = (rng.permutation(n_slab) + 0.5) / n_slab * (L / slab)
    x0 = (np.repeat(base, slab) + np.tile(np.arange(slab), n_slab) * (L / slab)) % L
    x = (x0 - amp / k * np.sin(k * x0)) % L
    cell, off = _split(x / dx, n_cells)
    vy = vt * rng.standard_normal(N)
    vz = vt * rng.standard_normal(N)
    cfg = dict(
        name=f"langmuir_klD{k_lambda_d}", periodic=1, n_cells=n_cells, length=L, dt=wpdt / wp,
        bg_charge=E_CHARGE * n0, species=[dict(q=-E_CHARGE, m=M_E, w=n0 * L / N)],
        seed=seed, diag_interval=0,
        info=dict(omega_p=wp, lambda_d=lam_d, k=k, n0=n0, te_ev=te_ev),
    )
    parts = [dict(cell=cell, off=off, vx=vx.astype(np.float32), vy=vy.astype(np.float32),
                  vz=vz.astype(np.float32), id=np.arange(N, dtype=np.uint32))]
    return cfg, parts


def ccp_case(seed: int = 1, n_cells: int = 512, gap: float = 0.025, n_per_species: int = 200_000,
             volts: float = 200.0, freq: float = 13.56e6, mtorr: float = 30.0, n0: float = 2e14,
             te_ev: float = 2.0, steps_per_cycle: int = 400, see_gamma: float = 0.1, harmonics=None):
    """Single-frequency argon CCP with the synthetic argon tables: uniform
    plasma of density n0 between two electrodes, Maxwellian electrons at
    te_ev and ions at the gas temperature (300 K)."""
    tg = 300.0
    ng = mtorr * 1e-3 * TORR / (K_B * tg)
    w = n0 * gap / n_per_species
    rng = np.random.default_rng(seed)
    e = maxwellian_load(rng, n_per_species, n_cells, te_ev, M_E)
    i = maxwellian_load(rng, n_per_species, n_cells, K_B * tg / E_CHARGE, M_AR)
    cfg = dict(
        name="argon_ccp", periodic=0, n_cells=n_cells, length=gap, dt=1.0 / (freq * steps_per_cycle),
        gas_density=ng, gas_temp=tg, gas_mass=M_AR,
        harmonics=harmonics if harmonics is not None else [(freq, volts, 0.0)],
        see_gamma=see_gamma, see_temp_ev=1.0,
        species=[dict(q=-E_CHARGE, m=M_E, w=w), dict(q=E_CHARGE, m=M_AR, w=w)],
        xsec=argon_tables(), seed=seed, diag_interval=0,
    )
    return cfg, [e, i]


def ecdi_case(seed: int = 1, n_cells: int = 2048, ppc: int = 2500, length: float = 5e-3,
              n0: float = 1e17, B: float = 0.02, E: float = 2e4, te_ev: float = 10.0,
              ti_ev: float = 0.5, dt: float = 5e-12, nu: float = 1e6):
    """E x B azimuthal box of a Hall thruster (paper §3.6: xenon, 1e17 m^-3,
    B = 200 G, E = 20 kV/m): x azimuthal and periodic, E_ext along z, B along
    y, so the electrons drift at v_E = -E/B along x; they are loaded as a
    Maxwellian drifting at v_E; the ions at rest.  Electron-neutral
    collisions use a constant frequency nu (elastic, isotropic, xenon recoil)."""
    N = n_cells * ppc
    w = n0 * length / N
    rng = np.random.default_rng(seed)
    e = maxwellian_load(rng, N, n_cells, te_ev, M_E, drift=(-E / B, 0.0, 0.0))
    i = maxwellian_load(rng, N, n_cells, ti_ev, M_XE)
    cfg = dict(
        name="ecdi_exb", periodic=1, n_cells=n_cells, length=length, dt=dt,
        gas_density=0.0, gas_temp=300.0, gas_mass=M_XE, B=(0.0, B, 0.0), E_ext=(0.0, 0.0, E),
        const_nu_e=nu,
        species=[dict(q=-E_CHARGE, m=M_E, w=w), dict(q=E_CHARGE, m=M_XE, w=w)],
        seed=seed, diag_interval=0,
    )
    return cfg, [e, i]


def sweep_cases(n_cases: int = 256, seed: int = 2609, freq: float = 13.56e6, n0: float = 2e14,
                n_range=(5e4, 1e6), steps_per_cycle: int = 1600):
    """Parameter sweep of argon CCPs (uneven sizes): pressure 10-300 mTorr,
    voltage 100-500 V, gap 2-6 cm, 256-2048 cells, 5e4-1e6 particles per
    species, drawn with numpy's Philox bit generator.  Returns the case
    descriptions and, per case, the particle count per species; the
    particles themselves are sampled on the device (uniform density n0,
    electrons 2 eV, ions at 300 K).  The drive is V0 sin(2 pi f t): it starts
    at zero, so the plasma shields the electrodes as the voltage rises
    instead of meeting the full vacuum field at t = 0.  The step is 1/1600 of
    the period: at 1/400 the densest cases (300 mTorr, 500 V) ionize until
    omega_pe dt passes the leapfrog limit of 2 (near 3e16 m^-3) within a few
    periods, and then grow without bound."""
    rng = np.random.Generator(np.random.Philox(seed))
    cfgs, counts = [], []
    tables = argon_tables()
    for i in range(n_cases):
        mtorr = rng.uniform(10.0, 300.0)
        volts = rng.uniform(100.0, 500.0)
        gap = rng.uniform(0.02, 0.06)
        n_cells = int(rng.integers(256, 2049))
        n = int(rng.uniform(*n_range))
        tg = 300.0
        cfg = dict(
            name=f"sweep_{i}", periodic=0, n_cells=n_cells, length=gap, dt=1.0 / (freq * steps_per_cycle),
            gas_density=mtorr * 1e-3 * TORR / (K_B * tg), gas_temp=tg, gas_mass=M_AR,
            harmonics=[(freq, volts, -0.5 * math.pi)], see_gamma=0.1, see_temp_ev=1.0,
            species=[dict(q=-E_CHARGE, m=M_E, w=n0 * gap / n), dict(q=E_CHARGE, m=M_AR, w=n0 * gap / n)],
            xsec=tables, seed=seed * 1000 + i, diag_interval=0,
            load=dict(n=n, n0=n0, te_ev=2.0, ti_ev=K_B * tg / E_CHARGE),
        )
        cfgs.append(cfg)
        counts.append(n)
    return cfgs, counts


def dual_frequency_family(n_cases: int, seed: int, n_cells: int = 256, gap: float = 0.03, n0: float = 2e14,
                          n_init: int = 2500, freq: float = 13.56e6, steps_per_cycle: int = 1600):
    """Dual-frequency argon CCPs, V(t) = V1 cos(2 pi f t + theta) + V2 cos(4 pi f t)
    (the two-harmonic waveform of the paper's §3.3), drawn with numpy's Philox:
    p in [10, 100] mTorr, V1, V2 in [50, 300] V, theta in [0, 90 deg], 3 cm gap.
    These discharges reach 1e16 - 2e16 m^-3 with the synthetic tables, so the
    step is 1/1600 of the period (omega_pe dt <= 0.4 there; 400 steps per
    period would put omega_pe dt near the leapfrog limit of 2).
    Returns (cfgs, params) with params[i] = (p_mTorr, V1, V2, theta)."""
    rng = np.random.Generator(np.random.Philox(seed))
    tables = argon_tables()
    cfgs, params = [], []
    tg = 300.0
    w = n0 * gap / n_init
    for i in range(n_cases):
        mtorr = rng.uniform(10.0, 100.0)
        v1, v2 = rng.uniform(50.0, 300.0), rng.uniform(50.0, 300.0)
        theta = rng.uniform(0.0, 0.5 * math.pi)
        cfgs.append(dict(
            name=f"dual_freq_{seed}_{i}", periodic=0, n_cells=n_cells, length=gap, dt=1.0 / (freq * steps_per_cycle),
            gas_density=mtorr * 1e-3 * TORR / (K_B * tg), gas_temp=tg, gas_mass=M_AR,
            harmonics=[(freq, v1, theta), (2 * freq, v2, 0.0)], see_gamma=0.1, see_temp_ev=1.0,
            species=[dict(q=-E_CHARGE, m=M_E, w=w), dict(q=E_CHARGE, m=M_AR, w=w)],
            xsec=tables, seed=seed * 1000 + i, diag_interval=8,
            load=dict(n=n_init, n0=n0, te_ev=2.0, ti_ev=K_B * tg / E_CHARGE),
        ))
        params.append((mtorr, v1, v2, theta))
    return cfgs, np.array(params)
