"""FP64 CPU oracle of the 1D3V electrostatic PIC-MCC step (ctypes wrapper).

TEST INFRASTRUCTURE.  This package is the oracle: only ``tests/``,
``__graft_entry__.smoke()`` and ``bench.py``'s CPU legs may import it.  The
CUDA library never loads it and it never loads the CUDA library.

The C source (``pic_oracle.c``) restates the method of the paper (§1:
explicit leapfrog, Boris pusher, null-collision Monte Carlo with tabulated
cross sections, walls with secondary emission, Poisson's equation) one
particle at a time in FP64.  ``build()`` compiles it with gcc; importing this
module builds it when the shared object is missing or older than its source.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pic_oracle.c")
_HDR = os.path.join(_HERE, "pic_oracle.h")
_LIB = os.path.join(_HERE, "liboracle.so")

NGRID = 1000
EEPF_BINS = 240
IFEDF_BINS = 256
ELASTIC, EXCITATION, IONIZATION, ISO, CX = 0, 1, 2, 3, 4


def build(force: bool = False) -> str:
    """Compile the oracle into ``oracle/liboracle.so`` (plain -O2, single thread)."""
    newest = max(os.path.getmtime(_SRC), os.path.getmtime(_HDR))
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < newest:
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-D_GNU_SOURCE", "-fPIC", "-shared",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


class Params(C.Structure):
    _fields_ = [
        ("periodic", C.c_int32), ("n_cells", C.c_int32),
        ("length", C.c_double), ("dt", C.c_double),
        ("gas_density", C.c_double), ("gas_temp", C.c_double), ("gas_mass", C.c_double),
        ("B", C.c_double * 3), ("E_ext", C.c_double * 3),
        ("n_harm", C.c_int32),
        ("harm_freq", C.c_double * 4), ("harm_amp", C.c_double * 4), ("harm_phase", C.c_double * 4),
        ("see_gamma", C.c_double), ("see_temp_ev", C.c_double),
        ("bg_charge", C.c_double), ("const_nu_e", C.c_double),
        ("n_species", C.c_int32),
        ("q", C.c_double * 2), ("m", C.c_double * 2), ("w", C.c_double * 2),
        ("seed", C.c_uint64),
        ("diag_interval", C.c_int32), ("rewind", C.c_int32),
        ("circuit", C.c_int32), ("cap", C.c_double), ("ifedf_emax_ev", C.c_double),
        ("no_field", C.c_int32),
        ("axial_len", C.c_double), ("renew_temp_ev", C.c_double * 2), ("renew_drift", (C.c_double * 3) * 2),
    ]


class Counters(C.Structure):
    _fields_ = [
        ("n_steps", C.c_int64), ("n_diag", C.c_int64),
        ("absorbed", (C.c_int64 * 2) * 2), ("see_emitted", C.c_int64),
        ("candidates", C.c_int64 * 2), ("collisions", (C.c_int64 * 4) * 2),
        ("ionizations", C.c_int64), ("step", C.c_int64), ("renewed", C.c_int64 * 2),
    ]


def _load():
    lib = C.CDLL(build())
    P = C.c_void_p
    dp = C.POINTER(C.c_double)
    lib.or_create.restype = P
    lib.or_create.argtypes = [C.POINTER(Params)]
    lib.or_destroy.argtypes = [P]
    lib.or_load_xsec.argtypes = [P, C.c_int, C.c_int, C.c_double, dp, dp, C.c_int]
    lib.or_load_particles.argtypes = [P, C.c_int, C.c_int64, dp, dp, dp, dp, C.POINTER(C.c_uint32)]
    lib.or_step.argtypes = [P, C.c_int64]
    lib.or_load_profile.argtypes = [P, C.c_int, C.c_int64, dp, dp, dp, C.c_uint32]
    lib.or_count.restype = C.c_int64
    lib.or_count.argtypes = [P, C.c_int]
    lib.or_get_particles.argtypes = [P, C.c_int, dp, dp, dp, dp, C.POINTER(C.c_uint32), dp,
                                     C.POINTER(C.c_int32)]
    lib.or_get_field.argtypes = [P, dp, dp]
    lib.or_get_axial.argtypes = [P, C.c_int, dp]
    lib.or_get_clock.argtypes = [P, C.c_int, C.POINTER(C.c_int32)]
    lib.or_get_loss_speed.argtypes = [P, C.c_int, dp]
    lib.or_get_move.argtypes = [P, C.c_int, dp]
    lib.or_neg_log_u32.restype = C.c_float
    lib.or_neg_log_u32.argtypes = [C.c_float]
    lib.or_clock_state.restype = C.c_int32
    lib.or_clock_state.argtypes = [C.c_float, C.c_float, dp]
    lib.or_get_deposit.argtypes = [P, C.c_int, C.POINTER(C.c_int64)]
    lib.or_get_numax.argtypes = [P, C.c_int, dp]
    lib.or_get_nu_table.argtypes = [P, C.c_int, C.c_int, dp]
    lib.or_get_counters.argtypes = [P, C.POINTER(Counters)]
    lib.or_get_moments.argtypes = [P, dp, dp, dp, dp, dp, dp, dp]
    lib.or_reset_moments.argtypes = [P]
    lib.or_get_ifedf.argtypes = [P, dp]
    lib.or_get_electrode_charge.restype = C.c_double
    lib.or_get_electrode_charge.argtypes = [P]
    lib.or_get_field_energy.restype = C.c_int64
    lib.or_get_field_energy.argtypes = [P, dp, C.c_int64]
    lib.or_philox4x32_10.argtypes = [C.POINTER(C.c_uint32), C.POINTER(C.c_uint32), C.POINTER(C.c_uint32)]
    lib.or_uniform.restype = C.c_double
    lib.or_uniform.argtypes = [C.c_uint32]
    lib.or_deposit.argtypes = [C.c_int, C.c_int, C.c_int64, dp, C.POINTER(C.c_int64)]
    lib.or_poisson.argtypes = [C.c_int, C.c_int, C.c_double, dp, C.c_double, dp]
    lib.or_boris.argtypes = [C.c_double, C.c_double, dp, dp, dp]
    lib.or_sort_by_cell.restype = C.c_int64
    lib.or_sort_by_cell.argtypes = [C.c_int, C.c_int64, C.POINTER(C.c_int32), C.POINTER(C.c_int64)]
    return lib


_lib = _load()


def _d(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


# --------------------------------------------------------------------------- primitives
def philox4x32_10(ctr, key):
    """Philox4x32-10 of one counter (4 uint32) under one key (2 uint32)."""
    c = (C.c_uint32 * 4)(*[int(x) & 0xFFFFFFFF for x in ctr])
    k = (C.c_uint32 * 2)(*[int(x) & 0xFFFFFFFF for x in key])
    o = (C.c_uint32 * 4)()
    _lib.or_philox4x32_10(c, k, o)
    return [int(x) for x in o]


def uniform(r: int) -> float:
    return float(_lib.or_uniform(C.c_uint32(int(r) & 0xFFFFFFFF)))


CLOCK_MAX = 131071


def neg_log_u32(u: float) -> float:
    """-ln(u) as the collision clock computes it (FP32)."""
    return float(_lib.or_neg_log_u32(C.c_float(u)))


def clock_state(u: float, lam: float) -> int:
    """Clock state 2 k + c of a fresh gap from uniform u, lam = numax dt (both FP32)."""
    return int(_lib.or_clock_state(C.c_float(u), C.c_float(lam), None))


def deposit(n_cells: int, periodic: bool, xi) -> np.ndarray:
    """Raw CIC deposit (units of 2^-32 particle) of positions xi (cell units)."""
    xi = _f64(xi)
    nn = n_cells if periodic else n_cells + 1
    R = np.zeros(nn, dtype=np.int64)
    _lib.or_deposit(n_cells, int(bool(periodic)), xi.size, _d(xi), R.ctypes.data_as(C.POINTER(C.c_int64)))
    return R


def poisson(n_cells: int, periodic: bool, dx: float, rho, phi_left: float = 0.0) -> np.ndarray:
    rho = _f64(rho)
    phi = np.zeros_like(rho)
    _lib.or_poisson(n_cells, int(bool(periodic)), dx, _d(rho), phi_left, _d(phi))
    return phi


def boris(qm: float, h: float, E, B, v) -> np.ndarray:
    E = _f64(E); B = _f64(B); v = _f64(v).copy()
    _lib.or_boris(qm, h, _d(E), _d(B), _d(v))
    return v


def sort_by_cell(n_cells: int, cell) -> np.ndarray:
    """Indices of the particles with a cell in [0, n_cells), grouped by ascending
    cell, input order kept inside a cell (counting sort)."""
    cell = np.ascontiguousarray(cell, dtype=np.int32)
    perm = np.zeros(cell.size, dtype=np.int64)
    k = _lib.or_sort_by_cell(n_cells, cell.size, cell.ctypes.data_as(C.POINTER(C.c_int32)),
                             perm.ctypes.data_as(C.POINTER(C.c_int64)))
    return perm[:k]


# --------------------------------------------------------------------------- case
def make_params(cfg: dict) -> Params:
    """Fill the oracle's parameter block from a workload description dict."""
    p = Params()
    p.periodic = int(cfg["periodic"])
    p.n_cells = int(cfg["n_cells"])
    p.length = float(cfg["length"])
    p.dt = float(cfg["dt"])
    p.gas_density = float(cfg.get("gas_density", 0.0))
    p.gas_temp = float(cfg.get("gas_temp", 300.0))
    p.gas_mass = float(cfg.get("gas_mass", 1.0))
    for i in range(3):
        p.B[i] = float(cfg.get("B", (0, 0, 0))[i])
        p.E_ext[i] = float(cfg.get("E_ext", (0, 0, 0))[i])
    harm = cfg.get("harmonics", [])
    p.n_harm = len(harm)
    for i, (f, a, ph) in enumerate(harm):
        p.harm_freq[i], p.harm_amp[i], p.harm_phase[i] = f, a, ph
    p.see_gamma = float(cfg.get("see_gamma", 0.0))
    p.see_temp_ev = float(cfg.get("see_temp_ev", 1.0))
    p.bg_charge = float(cfg.get("bg_charge", 0.0))
    p.const_nu_e = float(cfg.get("const_nu_e", 0.0))
    sp = cfg["species"]
    p.n_species = len(sp)
    for i, s in enumerate(sp):
        p.q[i], p.m[i], p.w[i] = s["q"], s["m"], s["w"]
    p.seed = int(cfg.get("seed", 0)) & 0xFFFFFFFFFFFFFFFF
    p.diag_interval = int(cfg.get("diag_interval", 0))
    p.rewind = int(cfg.get("rewind", 1))
    p.circuit = {"voltage": 0, "capacitor": 1, "current": 2}[cfg.get("circuit", "voltage")]
    p.cap = float(cfg.get("blocking_cap", 0.0))
    p.ifedf_emax_ev = float(cfg.get("ifedf_emax_ev", 0.0))
    p.no_field = int(bool(cfg.get("no_field", False)))
    p.axial_len = float(cfg.get("axial_length", 0.0))
    for i, s in enumerate(sp):
        p.renew_temp_ev[i] = float(s.get("renew_temp_ev", 0.0))
        for k in range(3):
            p.renew_drift[i][k] = float(s.get("renew_drift", (0.0, 0.0, 0.0))[k])
    return p


class Case:
    """One oracle simulation: ``Case(cfg)``, ``load_xsec``, ``load_particles``, ``step``."""

    def __init__(self, cfg: dict):
        self.cfg = cfg
        self._p = make_params(cfg)
        self._h = _lib.or_create(C.byref(self._p))
        if not self._h:
            raise ValueError("oracle rejected the case parameters")
        self.n_cells = int(cfg["n_cells"])
        self.periodic = bool(cfg["periodic"])
        self.n_nodes = self.n_cells if self.periodic else self.n_cells + 1
        for t in cfg.get("xsec", []):
            self.load_xsec(t["species"], t["kind"], t["threshold"], t["energy"], t["sigma"])

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            _lib.or_destroy(h)
            self._h = None

    def load_xsec(self, sp, kind, threshold, energy, sigma):
        e = _f64(energy); s = _f64(sigma)
        if _lib.or_load_xsec(self._h, sp, kind, threshold, _d(e), _d(s), e.size) != 0:
            raise ValueError("oracle rejected a cross-section table")

    def load_particles(self, sp, xi, vx, vy, vz, ids):
        xi, vx, vy, vz = _f64(xi), _f64(vx), _f64(vy), _f64(vz)
        ids = np.ascontiguousarray(ids, dtype=np.uint32)
        rc = _lib.or_load_particles(self._h, sp, xi.size, _d(xi), _d(vx), _d(vy), _d(vz),
                                    ids.ctypes.data_as(C.POINTER(C.c_uint32)))
        if rc != 0:
            raise ValueError(f"oracle rejected the particles ({rc})")

    def load_profile(self, sp, n, density, temp_ev, drift=(0.0, 0.0, 0.0), id_base=0):
        d = _f64(density); t = _f64(temp_ev); dr = _f64(drift)
        if _lib.or_load_profile(self._h, sp, int(n), _d(d), _d(t), _d(dr), int(id_base) & 0xFFFFFFFF) != 0:
            raise ValueError("oracle rejected the profile load")

    def step(self, n=1):
        if _lib.or_step(self._h, int(n)) != 0:
            raise RuntimeError("oracle step failed")

    def count(self, sp):
        return int(_lib.or_count(self._h, sp))

    def particles(self, sp) -> dict:
        n = self.count(sp)
        out = {k: np.zeros(n) for k in ("xi", "vx", "vy", "vz", "margin")}
        out["id"] = np.zeros(n, dtype=np.uint32)
        out["event"] = np.zeros(n, dtype=np.int32)
        _lib.or_get_particles(self._h, sp, _d(out["xi"]), _d(out["vx"]), _d(out["vy"]), _d(out["vz"]),
                              out["id"].ctypes.data_as(C.POINTER(C.c_uint32)), _d(out["margin"]),
                              out["event"].ctypes.data_as(C.POINTER(C.c_int32)))
        out["vloss"] = np.zeros(n)          # speed before a threshold loss in the last step (0: none)
        _lib.or_get_loss_speed(self._h, sp, _d(out["vloss"]))
        out["xmove"] = np.zeros(n)          # cells of the move that placed it in the last step
        _lib.or_get_move(self._h, sp, _d(out["xmove"]))
        return out

    def clock(self, sp) -> np.ndarray:
        """Collision clock 2 k + c of each particle, in the order of ``particles``."""
        out = np.zeros(self.count(sp), dtype=np.int32)
        _lib.or_get_clock(self._h, sp, out.ctypes.data_as(C.POINTER(C.c_int32)))
        return out

    def axial(self, sp) -> np.ndarray:
        """Axial excursion z (m) of each particle, in the order of ``particles``."""
        z = np.zeros(self.count(sp))
        _lib.or_get_axial(self._h, sp, _d(z))
        return z

    def field(self):
        phi = np.zeros(self.n_nodes); E = np.zeros(self.n_nodes)
        _lib.or_get_field(self._h, _d(phi), _d(E))
        return phi, E

    def deposit(self, sp):
        R = np.zeros(self.n_nodes, dtype=np.int64)
        _lib.or_get_deposit(self._h, sp, R.ctypes.data_as(C.POINTER(C.c_int64)))
        return R

    def numax(self, sp):
        v = C.c_double()
        _lib.or_get_numax(self._h, sp, C.byref(v))
        return v.value

    def nu_table(self, sp, k):
        nu = np.zeros(NGRID)
        if _lib.or_get_nu_table(self._h, sp, k, _d(nu)) != 0:
            raise IndexError(k)
        return nu

    def counters(self) -> dict:
        c = Counters()
        _lib.or_get_counters(self._h, C.byref(c))
        return {
            "n_steps": c.n_steps, "n_diag": c.n_diag,
            "absorbed": np.array([[c.absorbed[s][w] for w in range(2)] for s in range(2)]),
            "see_emitted": c.see_emitted,
            "candidates": np.array([c.candidates[s] for s in range(2)]),
            "collisions": np.array([[c.collisions[s][k] for k in range(4)] for s in range(2)]),
            "ionizations": c.ionizations, "step": c.step, "renewed": np.array(list(c.renewed)),
        }

    def moments(self) -> dict:
        nn = self.n_nodes
        dens = np.zeros(2 * nn); phi = np.zeros(nn); en = np.zeros(2 * nn); dd = np.zeros(2 * nn)
        eepf = np.zeros(EEPF_BINS); ke = np.zeros(2); pw = np.zeros(2)
        _lib.or_get_moments(self._h, _d(dens), _d(phi), _d(en), _d(dd), _d(eepf), _d(ke), _d(pw))
        return {"dens_sum": dens.reshape(2, nn), "phi_sum": phi, "en_sum": en.reshape(2, nn),
                "dens_diag_sum": dd.reshape(2, nn), "eepf": eepf, "ke_sum": ke, "pw_sum": pw}

    def reset_moments(self):
        _lib.or_reset_moments(self._h)

    def ifedf(self) -> np.ndarray:
        """Ion energy histogram at each electrode, shape (2, IFEDF_BINS)."""
        out = np.zeros(2 * IFEDF_BINS)
        _lib.or_get_ifedf(self._h, _d(out))
        return out.reshape(2, IFEDF_BINS)

    def electrode_charge(self) -> float:
        """Charge per area of electrode 0 with its capacitor plate (C/m^2)."""
        return float(_lib.or_get_electrode_charge(self._h))

    def field_energy(self) -> np.ndarray:
        n = int(_lib.or_get_field_energy(self._h, None, 0))
        out = np.zeros(n)
        _lib.or_get_field_energy(self._h, _d(out), n)
        return out
