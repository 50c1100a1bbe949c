"""GPU parity of the parts a one-step particle comparison does not reach: the
FP64 field solve on identical charge, the diagnostic moments bin by bin, the
network's Adam update and the warm-start loader, the SI-unit particle load,
and the error paths (a device wait that gives up, a non-finite field).  All
calls go through the C ABI; the expected values come from the oracle."""
import numpy as np
import pytest

from paper_2609_17151_b300 import workloads as W

from .gpu_helpers import compare_species, gpu_case, oracle_case

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA device", allow_module_level=True)

import oracle  # noqa: E402
from oracle import mlp as omlp  # noqa: E402
from paper_2609_17151_b300 import pic  # noqa: E402

ELEM = 1.602176634e-19


def small_ccp(seed=3, n=20001, te=20.0, ti_ev=400.0, n_cells=64, volts=200.0):
    gap = n_cells * (0.025 / 512)
    cfg, parts = W.ccp_case(seed=seed, n_cells=n_cells, gap=gap, n_per_species=n, te_ev=te, volts=volts,
                            see_gamma=0.5)
    if ti_ev is not None:
        rng = np.random.default_rng(seed + 100)
        parts[1] = W.maxwellian_load(rng, n, n_cells, ti_ev, W.M_AR)
    return cfg, parts


# --------------------------------------------------------------------------- FP64 field solve
@pytest.mark.parametrize("which", ["ccp_512", "langmuir_64", "exb_2048"])
def test_field_solve_matches_oracle_at_fp64(which):
    """The exact-integer prefix-sum solve on the GPU (paper §1's Poisson
    equation) against the oracle's Thomas solve on the same deposit: the raw
    deposits are bit-identical, phi and E agree to 1e-12 of their largest
    value (both FP64; the two differ only in rounding order)."""
    if which == "ccp_512":
        cfg, parts = W.ccp_case(seed=5, n_per_species=200_000)
    elif which == "langmuir_64":
        cfg, parts = W.langmuir_case(seed=2)
    else:
        cfg, parts = W.ecdi_case(seed=3, ppc=20)
    oc = oracle_case(cfg, parts)
    oc.step(0)
    gc = gpu_case(cfg, parts)
    gc.step(0)
    phi_g, E_g, R_g = gc.field()
    phi_o, E_o = oc.field()
    for s in range(len(cfg["species"])):
        assert np.array_equal(R_g[s], oc.deposit(s)), s
    assert np.abs(phi_g - phi_o).max() <= 1e-12 * np.abs(phi_o).max()
    assert np.abs(E_g - E_o).max() <= 1e-12 * np.abs(E_o).max()
    gc.close()


# --------------------------------------------------------------------------- diagnostics
def _eepf_bins(p, mass, n_cells):
    """EEPF bin of each electron of the central 10 % of the gap (paper §3.2
    reading: 0.25 eV bins), -1 outside."""
    xi = p["cell"].astype(np.float64) + p["off"] if "cell" in p else p["xi"]
    v2 = p["vx"].astype(np.float64) ** 2 + p["vy"].astype(np.float64) ** 2 + p["vz"].astype(np.float64) ** 2
    eps = 0.5 * mass * v2 / ELEM
    b = np.floor(eps / 0.25).astype(np.int64)
    inside = (xi >= 0.45 * n_cells) & (xi < 0.55 * n_cells) & (b < 240)
    return np.where(inside, b, -1)


def test_eepf_bin_by_bin_and_power_sum_match_oracle():
    """After one diagnostic step the GPU's EEPF equals the oracle's bin by
    bin except for electrons whose energy falls in different bins on the two
    sides (matched by id, at most those), and the J.E sum agrees to FP32
    accumulation of FP32 particle state."""
    cfg, parts = small_ccp(seed=21, n=60_001, te=15.0)
    cfg["diag_interval"] = 1
    oc = oracle_case(cfg, parts)
    oc.step(0)
    E0 = oc.field()[1]
    oc.step(1)
    gc = gpu_case(cfg, parts)
    gc.step(1)
    mg, mo = gc.moments(), oc.moments()
    g, o = gc.particles(0), oc.particles(0)
    me = cfg["species"][0]["m"]
    bg, bo = _eepf_bins(g, me, cfg["n_cells"]), _eepf_bins(o, me, cfg["n_cells"])
    ig, io = np.argsort(g["id"], kind="stable"), np.argsort(o["id"], kind="stable")
    assert np.array_equal(g["id"][ig], o["id"][io])
    flips = int(np.sum(bg[ig] != bo[io]))
    # the kernel bins in FP32: electrons within FP32 rounding of a bin or
    # region edge may land on either side of it
    xg = g["cell"].astype(np.float64) + g["off"]
    eg = 0.5 * me * (g["vx"].astype(np.float64) ** 2 + g["vy"].astype(np.float64) ** 2
                     + g["vz"].astype(np.float64) ** 2) / ELEM / 0.25
    n = cfg["n_cells"]
    edge = ((np.abs(eg - np.round(eg)) < 1e-5 * np.maximum(eg, 1.0))
            | (np.abs(xg - 0.45 * n) < 1e-4) | (np.abs(xg - 0.55 * n) < 1e-4))
    allowed = flips + int(edge.sum())
    assert allowed <= 5e-3 * bg.size
    d = np.abs(mg["eepf"] - mo["eepf"])
    assert d.sum() <= 2 * allowed, (d.sum(), flips, int(edge.sum()))
    assert mg["eepf"].sum() > 1000
    # J.E: sum over particles of q w v_x^{1/2} E^0(x^0), per species
    dx = cfg["length"] / cfg["n_cells"]
    for s in range(2):
        sp = cfg["species"][s]
        xi0 = W.as_xi(parts[s])
        j = np.floor(xi0).astype(int)
        t = xi0 - j
        e_at = (1 - t) * E0[j] + t * E0[np.minimum(j + 1, E0.size - 1)]
        scale = abs(sp["q"]) * sp["w"] * np.sum(np.abs(e_at) * np.abs(parts[s]["vx"].astype(np.float64)))
        assert abs(mg["pw_sum"][s] - mo["pw_sum"][s]) <= 2e-5 * scale + 1e-12, (s, mg["pw_sum"][s], mo["pw_sum"][s])
    assert dx > 0
    gc.close()


# --------------------------------------------------------------------------- collision clock
@pytest.mark.parametrize("which", ["ccp_hot", "exb_const_nu"])
def test_collision_clocks_are_bit_identical_to_the_oracle(which):
    """The null-collision clock of every particle (steps left to its next
    collision candidate, drawn in FP32 from the same Philox words on both
    sides) is the same integer on the GPU and in the oracle after several
    steps, for the table-driven argon CCP (every process, products with their
    first clocks) and the constant-frequency E x B electrons."""
    if which == "ccp_hot":
        cfg, parts = small_ccp(seed=31, n=30_001, te=25.0)
        steps = 6
    else:
        cfg, parts = W.ecdi_case(seed=5, ppc=20, nu=2e9)
        steps = 4
    oc = oracle_case(cfg, parts)
    oc.step(steps)
    gc = gpu_case(cfg, parts)
    gc.step(steps)
    for s in range(len(cfg["species"])):
        g, o = gc.particles(s), oc.particles(s)
        cg, co = gc.clock(s), oc.clock(s)
        ig, io = np.argsort(g["id"], kind="stable"), np.argsort(o["id"], kind="stable")
        assert np.array_equal(g["id"][ig], o["id"][io])
        assert np.array_equal(cg[ig].astype(np.int64), co[io].astype(np.int64)), s
        if s == 0:
            assert np.any(cg % 2 == 0) and np.unique(cg).size > 10
    gc.close()


# --------------------------------------------------------------------------- network
def test_gpu_adam_matches_oracle_adam_over_ten_steps():
    """pic_mlp_adam_step (the update pic_mlp_train applies) against the oracle's
    Adam on the same gradients: 10 steps from the same parameters agree to
    FP32 rounding (a wrong bias correction or moment decay moves them by
    about lr)."""
    net = pic.MLP(4, 32, 24, seed=3)
    p0 = net.params().astype(np.float64)
    rng = np.random.default_rng(8)
    p, m, v = p0.copy(), np.zeros_like(p0), np.zeros_like(p0)
    lr = 1e-3
    for t in range(1, 11):
        g = rng.normal(0.0, 1.0, p0.size) * rng.choice([1e-3, 1.0, 30.0], p0.size)
        g32 = g.astype(np.float32)
        net.adam_step(g32, lr)
        p, m, v = omlp.adam(p, g32.astype(np.float64), m, v, t, lr)
    pg = net.params().astype(np.float64)
    assert np.abs(pg - p).max() <= 1e-6 + 1e-6 * np.abs(p).max()
    assert np.abs(pg - p0).max() > 5e-3          # the parameters did move
    net.close()


def test_warmstart_train_equals_training_on_its_targets():
    """pic_warmstart_train builds the targets [log10 ne, log10 ni, Te] and the
    standardisation itself; training on them by hand gives the same network."""
    rng = np.random.default_rng(4)
    n_cases, n_points = 12, 16
    P = rng.uniform([10, 50, 50, 0], [100, 300, 300, 1.5], (n_cases, 4))
    x = np.linspace(0, 1, n_points)
    ne = 1e15 * (0.1 + np.sin(np.pi * x)[None, :] * P[:, :1] / 100)
    ni = 1.1 * ne
    te = 2 + P[:, 1:2] / 100 * (1 + x[None, :])
    lo, hi = np.array([10.0, 50, 50, 0]), np.array([100.0, 300, 300, 1.6])
    a = pic.MLP(4, 64, 3 * n_points, seed=5)
    ca = a.warmstart_train(P, ne, ni, te, lo, hi, epochs=200, lr=2e-3)
    Y = np.concatenate([np.log10(ne), np.log10(ni), te], 1).astype(np.float32).astype(np.float64)
    b = pic.MLP(4, 64, 3 * n_points, seed=5)
    b.set_normalization(lo, hi, Y.mean(0), Y.std(0) + 1e-3)
    cb = b.train(P, Y, epochs=200, lr=2e-3)
    assert ca[-1] < 0.05 * ca[0]
    assert np.allclose(ca, cb, rtol=1e-4, atol=1e-7)
    assert np.allclose(a.params(), b.params(), rtol=1e-4, atol=1e-6)
    a.close()
    b.close()


def test_warmstart_load_matches_oracle_restatement():
    """pic_warmstart_load: the network's prediction -> node profiles -> particle
    counts (restated in the oracle from the same prediction), then the
    profile loader (same ids and cells as the oracle's loader)."""
    n_points = 32
    cfg, _ = small_ccp(seed=61, n=10, n_cells=96)
    cfg["species"][0]["w"] = cfg["species"][1]["w"] = 4e8
    net = pic.MLP(4, 64, 3 * n_points, seed=9)
    mean = np.concatenate([np.full(n_points, 14.5), np.full(n_points, 14.6), np.full(n_points, 3.0)])
    net.set_normalization(np.zeros(4), np.ones(4), mean, np.full(3 * n_points, 0.05))
    prm = np.array([0.3, 0.7, 0.2, 0.9])
    y = net.predict(prm[None, :])[0]
    dx = cfg["length"] / cfg["n_cells"]
    w = (cfg["species"][0]["w"], cfg["species"][1]["w"])
    ne, ni, te, counts = omlp.warmstart_nodes(y, n_points, cfg["n_cells"], False, dx, w)
    assert min(counts) > 1000
    gc = pic.Case(cfg)
    gc.warmstart_load(net, prm, n_points, 0.03, id_base=11)
    assert list(gc.count()) == counts
    oc = oracle.Case(cfg)
    oc.load_profile(0, counts[0], ne, te, id_base=11)
    oc.load_profile(1, counts[1], ni, np.full(ne.size, 0.03), id_base=11)
    for s in range(2):
        g, o = gc.particles(s), oc.particles(s)
        ig, io = np.argsort(g["id"]), np.argsort(o["id"])
        assert np.array_equal(g["id"][ig], o["id"][io])
        cells_o = np.floor(o["xi"][io]).astype(np.int32)
        assert np.mean(g["cell"][ig] == cells_o) > 0.999
    gc.close()
    net.close()


# --------------------------------------------------------------------------- SI load
def test_si_load_is_bit_equal_to_the_cell_offset_load():
    """pic_load_particles_si converts x (m) and v (n x 3, m/s) on the device by
    the rule the header states; the same rule applied here and loaded through
    pic_load_particles gives bit-identical particles, on host and device input."""
    cfg, parts = small_ccp(seed=71, n=30_001)
    L, N = cfg["length"], cfg["n_cells"]
    dx = L / N
    rng = np.random.default_rng(3)
    n = 30_001
    x = rng.uniform(0, L, n)
    x[:4] = [0.0, np.nextafter(L, 0), dx * 17, dx * 17 * (1 - 1e-17)]
    v = rng.normal(0, 1e6, (n, 3))
    xi = x * (1.0 / dx)
    c = np.floor(xi)
    o = (xi - c).astype(np.float32)
    c = c.astype(np.int64)
    up = o >= np.float32(1.0)
    c[up] += 1
    o[up] = 0
    last = c >= N
    c[last] = N - 1
    o[last] = np.float32(0.99999994)
    ref = {"cell": c.astype(np.int32), "off": o, "vx": v[:, 0].astype(np.float32), "vy": v[:, 1].astype(np.float32),
           "vz": v[:, 2].astype(np.float32), "id": np.arange(n, dtype=np.uint32)}
    a = pic.Case(cfg)
    a.load(0, ref)
    b = pic.Case(cfg)
    b.load_si(0, x, v)
    d = pic.Case(cfg)
    d.load_si(0, torch.from_numpy(x).cuda(), torch.from_numpy(v.copy()).cuda(), on_device=True)
    pa = a.particles(0)
    for other in (b, d):
        pb = other.particles(0)
        for key in ("cell", "off", "vx", "vy", "vz", "id"):
            assert np.array_equal(pa[key], pb[key]), key
    # a position outside [0, L) is reported at the first step
    x[5] = L
    e = pic.Case(cfg)
    e.load_si(0, x, v)
    e.step(1)
    with pytest.raises(pic.PicError) as ei:
        e.sync()
    assert ei.value.status == 1
    for h in (a, b, d, e):
        h.close()


# --------------------------------------------------------------------------- error paths
def test_a_staging_wait_that_gives_up_reports_timeout_and_the_case_goes_on():
    """With a poll budget of 0 every staging wait of the step kernels gives up
    at once: the step reports PIC_ETIMEOUT (after waiting out the copies it
    issued), the context stays usable, and once the error is cleared and
    the budget restored the case steps normally."""
    cfg, parts = small_ccp(seed=81, n=20_001)
    gc = gpu_case(cfg, parts)
    gc.step(2)
    gc.sync()
    gc.set_wait_limit(0)
    gc.step(1)
    with pytest.raises(pic.PicError) as ei:
        gc.sync()
    assert ei.value.status == 6
    with pytest.raises(pic.PicError):           # sticky until cleared
        gc.sync()
    gc.clear_error()
    gc.set_wait_limit(1 << 22)
    gc.step(20)
    gc.sync()
    for s in range(2):
        p = gc.particles(s)
        assert p["id"].size > 0
        assert np.all(np.isfinite(p["vx"])) and np.all((p["off"] >= 0) & (p["off"] < 1))
        assert np.all((p["cell"] >= 0) & (p["cell"] < cfg["n_cells"]))
    x = torch.ones(1000, device="cuda")
    assert float(x.sum()) == 1000.0              # the context is healthy
    gc.close()


def test_non_finite_field_reports_numeric_error():
    """A finite background charge large enough that the FP64 Poisson source
    overflows gives a non-finite potential between two electrodes (a
    periodic box neutralises a uniform charge away): the field solve raises
    PIC_ENUMERIC (no particles are loaded, so nothing reads the field)."""
    cfg, parts = small_ccp(seed=2, n=10)
    cfg["bg_charge"] = 1.7e308
    empty = [{k: v[:0] for k, v in p.items()} for p in parts]
    gc = pic.Case(cfg, empty)
    gc.step(1)
    with pytest.raises(pic.PicError) as ei:
        gc.sync()
    assert ei.value.status == 5
    gc.close()


def test_one_step_parity_after_the_si_load():
    """The SI load feeds the same physics: one step from it matches the oracle
    loaded with the same positions."""
    cfg, parts = small_ccp(seed=91, n=8001)
    L, N = cfg["length"], cfg["n_cells"]
    xs, vs = [], []
    for p in parts:
        xs.append(W.as_xi(p) * (L / N))
        vs.append(np.stack([p["vx"], p["vy"], p["vz"]], 1).astype(np.float64))
    gc = pic.Case(cfg)
    for s in range(2):
        gc.load_si(s, xs[s], vs[s], parts[s]["id"])
    pg = [gc.particles(s) for s in range(2)]
    parts2 = [{"cell": q["cell"], "off": q["off"], "vx": q["vx"], "vy": q["vy"], "vz": q["vz"], "id": q["id"]}
              for q in pg]
    oc = oracle_case(cfg, parts2)
    oc.step(1)
    gc.step(1)
    dtdx = cfg["dt"] / (L / N)
    # velocities relative to at least 2 km/s: an ion all but stopped by an
    # isotropic centre-of-mass scatter carries the FP32 rounding of the ~30
    # km/s terms that formed it
    for s in range(2):
        compare_species(gc.particles(s), oc.particles(s), N, False, dtdx=dtdx, steps=1, vfloor=2e3)
    gc.close()
