"""Thin Python binding of the C ABI in ``include/pic1d3v.h`` (ctypes).

Argument marshalling only: every step of the method runs in the CUDA library
``libpic1d3v.so``.  Importing this module loads the library and raises if it
is missing (it is never replaced by anything else).  PyTorch, when present,
only supplies device memory (``torch_allocator``) and streams.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

ELASTIC, EXCITATION, IONIZATION, ISO, CX = 0, 1, 2, 3, 4
NGRID = 1000
EEPF_BINS = 240
MAX_PROC = 4
DESC_VERSION = 2
IFEDF_BINS = 256

STATUS = {0: "PIC_OK", 1: "PIC_EINVAL", 2: "PIC_ENOMEM", 3: "PIC_ECUDA", 4: "PIC_ECAPACITY",
          5: "PIC_ENUMERIC", 6: "PIC_ETIMEOUT", 7: "PIC_ESTATE"}

ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_size_t, C.c_void_p)


class CaseDesc(C.Structure):
    _fields_ = [
        ("struct_size", C.c_uint32), ("version", C.c_uint32),
        ("periodic", C.c_int32), ("n_cells", C.c_int32),
        ("length_m", C.c_double), ("dt_s", C.c_double),
        ("gas_density_m3", C.c_double), ("gas_temp_k", C.c_double), ("gas_mass_kg", C.c_double),
        ("B_T", C.c_double * 3), ("E_ext_V_per_m", C.c_double * 3),
        ("n_harm", C.c_int32),
        ("harm_freq_hz", C.c_double * 4), ("harm_amp_v", C.c_double * 4), ("harm_phase_rad", C.c_double * 4),
        ("see_gamma", C.c_double), ("see_temp_ev", C.c_double),
        ("background_charge_C_per_m3", C.c_double), ("const_nu_e_per_s", C.c_double),
        ("n_species", C.c_int32),
        ("charge_C", C.c_double * 2), ("mass_kg", C.c_double * 2), ("weight_per_m2", C.c_double * 2),
        ("capacity", C.c_int64 * 2),
        ("seed", C.c_uint64),
        ("sort_interval", C.c_int32), ("diag_interval", C.c_int32), ("rewind", C.c_int32),
        ("field_history", C.c_int32),
        ("circuit", C.c_int32), ("blocking_cap_F_per_m2", C.c_double), ("ifedf_emax_ev", C.c_double),
        ("no_field", C.c_int32),
        ("axial_length_m", C.c_double), ("renew_temp_ev", C.c_double * 2),
        ("renew_drift_m_per_s", (C.c_double * 3) * 2),
        ("stream", C.c_void_p),
        ("alloc", ALLOC_FN), ("free", FREE_FN), ("alloc_ctx", C.c_void_p),
    ]


class Moments(C.Structure):
    _fields_ = [
        ("struct_size", C.c_uint32), ("n_nodes", C.c_int32),
        ("step", C.c_int64), ("n_steps", C.c_int64), ("n_diag", C.c_int64),
        ("n_alive", C.c_int64 * 2), ("absorbed", (C.c_int64 * 2) * 2),
        ("see_emitted", C.c_int64), ("ionizations", C.c_int64),
        ("candidates", C.c_int64 * 2), ("collisions", (C.c_int64 * MAX_PROC) * 2),
        ("ke_sum", C.c_double * 2), ("pw_sum", C.c_double * 2),
        ("dens_sum", C.c_void_p), ("phi_sum", C.c_void_p), ("en_sum", C.c_void_p),
        ("dens_diag_sum", C.c_void_p), ("eepf", C.c_void_p),
        ("field_energy", C.c_void_p), ("field_energy_cap", C.c_int64), ("field_energy_n", C.c_int64),
        ("reset", C.c_int32), ("sort_interval", C.c_int32),
        ("ifedf", C.c_void_p), ("electrode_charge", C.c_double), ("renewed", C.c_int64 * 2),
    ]


class Tuning(C.Structure):
    _fields_ = [
        ("struct_size", C.c_uint32), ("tuned", C.c_int32), ("sort_interval", C.c_int32 * 2),
        ("threads", C.c_int32 * 2), ("stages", C.c_int32 * 2), ("grid", C.c_int32 * 2),
        ("shape_ms", (C.c_float * 6) * 2), ("sort_ms", C.c_float * 2), ("slope_ms", C.c_float * 2),
    ]


class KernelStat(C.Structure):
    _fields_ = [("name", C.c_char * 32), ("launches", C.c_int64), ("timed", C.c_int64), ("total_ms", C.c_double)]


class PicError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


def _load_library():
    path = _build.LIB
    if not os.path.exists(path):
        raise ImportError(f"CUDA library {path} is not built; run paper_2609_17151_b300/build.py")
    lib = C.CDLL(path)
    vp, i64, i32, dp = C.c_void_p, C.c_int64, C.c_int32, C.POINTER(C.c_double)
    lib.pic_create_case.argtypes = [C.POINTER(CaseDesc), C.POINTER(vp)]
    lib.pic_load_xsec_table.argtypes = [vp, C.c_int, C.c_int, C.c_double, dp, dp, C.c_int]
    lib.pic_load_particles.argtypes = [vp, C.c_int, i64, vp, vp, vp, vp, vp, vp, C.c_int]
    lib.pic_step.argtypes = [vp, i64]
    lib.pic_sync.argtypes = [vp]
    lib.pic_count.argtypes = [vp, C.POINTER(i64)]
    lib.pic_read_particles.argtypes = [vp, C.c_int, i64, C.POINTER(i64), vp, vp, vp, vp, vp, vp]
    lib.pic_read_field.argtypes = [vp, vp, vp, vp]
    lib.pic_read_axial.argtypes = [vp, C.c_int, i64, C.POINTER(i64), vp]
    lib.pic_read_clock.argtypes = [vp, C.c_int, i64, C.POINTER(i64), vp]
    lib.pic_read_moments.argtypes = [vp, C.POINTER(Moments)]
    lib.pic_read_tuning.argtypes = [vp, C.POINTER(Tuning)]
    lib.pic_set_step_shape.argtypes = [vp, C.c_int, C.c_int, C.c_int]
    lib.pic_checkpoint_size.argtypes = [vp, C.POINTER(C.c_uint64)]
    lib.pic_checkpoint_save.argtypes = [vp, vp, C.c_uint64]
    lib.pic_checkpoint_load.argtypes = [vp, vp, C.c_uint64]
    lib.pic_destroy.argtypes = [vp]
    lib.pic_status_str.restype = C.c_char_p
    lib.pic_status_str.argtypes = [C.c_int]
    lib.pic_last_error.restype = C.c_char_p
    lib.pic_philox.argtypes = [C.c_uint64, i64, vp, vp, vp]
    lib.pic_deposit.argtypes = [i32, i32, i64, vp, vp, vp, vp]
    lib.pic_sort_by_cell.argtypes = [i32, i64] + [vp] * 12 + [vp, vp]
    lib.pic_sort_by_cell_noalloc.argtypes = [i32, i64] + [vp] * 12 + [vp, vp]
    lib.pic_load_profile.argtypes = [vp, C.c_int, i64, dp, dp, dp, C.c_uint32]
    lib.pic_load_particles_si.argtypes = [vp, C.c_int, i64, vp, vp, vp, C.c_int]
    lib.pic_clear_error.argtypes = [vp]
    lib.pic_set_wait_limit.argtypes = [vp, C.c_uint32]
    lib.pic_batch_create.argtypes = [C.POINTER(CaseDesc), C.c_int, C.POINTER(vp)]
    lib.pic_batch_case.restype = vp
    lib.pic_batch_case.argtypes = [vp, C.c_int]
    lib.pic_batch_step.argtypes = [vp, i64]
    lib.pic_batch_sync.argtypes = [vp]
    lib.pic_batch_launches.restype = i64
    lib.pic_batch_launches.argtypes = [vp]
    lib.pic_batch_destroy.argtypes = [vp]
    lib.pic_batch_set_stages.argtypes = [vp, C.c_int]
    lib.pic_batch_set_own_threshold.argtypes = [vp, i64]
    lib.pic_batch_set_shape.argtypes = [vp, C.c_int]
    lib.pic_batch_tuning.argtypes = [vp, C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_int),
                                     C.POINTER(C.c_float), C.POINTER(C.c_float), C.POINTER(C.c_float)]
    lib.pic_batch_retune.argtypes = [vp]
    lib.pic_batch_freeze.argtypes = [vp, C.c_int, C.c_int]
    fp = C.POINTER(C.c_float)
    lib.pic_mlp_create.argtypes = [C.c_int, C.c_int, C.c_int, C.c_uint64, C.POINTER(vp)]
    lib.pic_mlp_set_normalization.argtypes = [vp, fp, fp, fp, fp]
    lib.pic_mlp_param_count.restype = i64
    lib.pic_mlp_param_count.argtypes = [vp]
    lib.pic_mlp_get_params.argtypes = [vp, fp]
    lib.pic_mlp_set_params.argtypes = [vp, fp]
    lib.pic_mlp_gradients.argtypes = [vp, fp, fp, C.c_int, fp, fp]
    lib.pic_mlp_train.argtypes = [vp, fp, fp, C.c_int, C.c_int, C.c_float, fp]
    lib.pic_mlp_predict.argtypes = [vp, fp, C.c_int, fp]
    lib.pic_mlp_adam_step.argtypes = [vp, fp, C.c_float]
    lib.pic_warmstart_train.argtypes = [vp, dp, dp, dp, dp, C.c_int, C.c_int, C.c_int, dp, dp, C.c_int, C.c_float,
                                        fp]
    lib.pic_mlp_destroy.argtypes = [vp]
    lib.pic_gemm_bf16.argtypes = [vp, C.c_int, C.c_int, vp, C.c_int, C.c_int, vp, C.c_int, C.c_int, C.c_int, C.c_int, vp]
    lib.pic_warmstart_load.argtypes = [vp, vp, dp, C.c_int, C.c_int, C.c_double, C.c_uint32, i64]
    lib.pic_profile.argtypes = [vp, C.c_int]
    lib.pic_profile_read.argtypes = [vp, C.POINTER(KernelStat), C.c_int, C.POINTER(C.c_int)]
    for f in ("pic_create_case", "pic_load_xsec_table", "pic_load_particles", "pic_step", "pic_sync", "pic_count",
              "pic_read_particles", "pic_read_field", "pic_read_moments", "pic_read_axial", "pic_read_tuning", "pic_set_step_shape", "pic_checkpoint_size",
              "pic_checkpoint_save", "pic_checkpoint_load", "pic_destroy", "pic_philox", "pic_deposit",
              "pic_profile", "pic_profile_read", "pic_sort_by_cell", "pic_sort_by_cell_noalloc",
              "pic_load_profile", "pic_batch_create", "pic_batch_step", "pic_batch_sync", "pic_batch_destroy",
              "pic_batch_set_stages", "pic_batch_set_own_threshold",
              "pic_mlp_create", "pic_mlp_set_normalization", "pic_mlp_get_params", "pic_mlp_set_params",
              "pic_mlp_gradients", "pic_mlp_train", "pic_mlp_predict", "pic_mlp_destroy", "pic_gemm_bf16",
              "pic_warmstart_load"):
        getattr(lib, f).restype = C.c_int
    return lib


lib = _load_library()


def check(status: int):
    if status != 0:
        raise PicError(status, lib.pic_last_error().decode(errors="replace"))


def _ptr(a) -> int | None:
    """Address of a numpy array or a torch tensor (None passes NULL)."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        return a.ctypes.data
    return a.data_ptr()


# --------------------------------------------------------------------------- torch plumbing
class TorchAllocator:
    """Device memory from PyTorch's caching allocator, handed to the library."""

    def __init__(self, device=None):
        import torch
        self._torch = torch
        self.device = torch.cuda.current_device() if device is None else device
        self._alloc = ALLOC_FN(self._do_alloc)
        self._free = FREE_FN(self._do_free)

    def _do_alloc(self, nbytes, ctx):
        try:
            return int(self._torch.cuda.caching_allocator_alloc(int(nbytes), self.device))
        except Exception:
            return None

    def _do_free(self, ptr, nbytes, ctx):
        self._torch.cuda.caching_allocator_delete(ptr)


# --------------------------------------------------------------------------- case
def make_desc(cfg: dict, *, stream=None, allocator: TorchAllocator | None = None,
              capacity=(0, 0), sort_interval: int = 0, field_history: int = 0) -> CaseDesc:
    d = CaseDesc()
    d.struct_size = C.sizeof(CaseDesc)
    d.version = DESC_VERSION
    d.periodic = int(cfg["periodic"])
    d.n_cells = int(cfg["n_cells"])
    d.length_m = float(cfg["length"])
    d.dt_s = float(cfg["dt"])
    d.gas_density_m3 = float(cfg.get("gas_density", 0.0))
    d.gas_temp_k = float(cfg.get("gas_temp", 300.0))
    d.gas_mass_kg = float(cfg.get("gas_mass", 1.0))
    for i in range(3):
        d.B_T[i] = float(cfg.get("B", (0, 0, 0))[i])
        d.E_ext_V_per_m[i] = float(cfg.get("E_ext", (0, 0, 0))[i])
    harm = cfg.get("harmonics", [])
    d.n_harm = len(harm)
    for i, (f, a, p) in enumerate(harm):
        d.harm_freq_hz[i], d.harm_amp_v[i], d.harm_phase_rad[i] = f, a, p
    d.see_gamma = float(cfg.get("see_gamma", 0.0))
    d.see_temp_ev = float(cfg.get("see_temp_ev", 1.0))
    d.background_charge_C_per_m3 = float(cfg.get("bg_charge", 0.0))
    d.const_nu_e_per_s = float(cfg.get("const_nu_e", 0.0))
    sp = cfg["species"]
    d.n_species = len(sp)
    for i, s in enumerate(sp):
        d.charge_C[i], d.mass_kg[i], d.weight_per_m2[i] = s["q"], s["m"], s["w"]
        d.capacity[i] = int(capacity[i]) if i < len(capacity) else 0
    d.seed = int(cfg.get("seed", 0)) & 0xFFFFFFFFFFFFFFFF
    d.sort_interval = int(cfg.get("sort_interval", sort_interval))
    d.diag_interval = int(cfg.get("diag_interval", 0))
    d.rewind = int(cfg.get("rewind", 1))
    d.field_history = int(field_history)
    d.circuit = {"voltage": 0, "capacitor": 1, "current": 2}[cfg.get("circuit", "voltage")]
    d.no_field = int(bool(cfg.get("no_field", False)))
    d.axial_length_m = float(cfg.get("axial_length", 0.0))
    for i, s in enumerate(cfg["species"]):
        d.renew_temp_ev[i] = float(s.get("renew_temp_ev", 0.0))
        for k in range(3):
            d.renew_drift_m_per_s[i][k] = float(s.get("renew_drift", (0.0, 0.0, 0.0))[k])
    d.blocking_cap_F_per_m2 = float(cfg.get("blocking_cap", 0.0))
    d.ifedf_emax_ev = float(cfg.get("ifedf_emax_ev", 0.0))
    d.stream = stream
    if allocator is not None:
        d.alloc, d.free = allocator._alloc, allocator._free
    return d


def create_case(desc: CaseDesc) -> int:
    h = C.c_void_p()
    check(lib.pic_create_case(C.byref(desc), C.byref(h)))
    return h.value


def load_xsec_table(h, species, kind, threshold_ev, energy_ev, sigma_m2):
    e = np.ascontiguousarray(energy_ev, dtype=np.float64)
    s = np.ascontiguousarray(sigma_m2, dtype=np.float64)
    check(lib.pic_load_xsec_table(h, species, kind, threshold_ev, e.ctypes.data_as(C.POINTER(C.c_double)),
                                  s.ctypes.data_as(C.POINTER(C.c_double)), e.size))


def load_particles(h, species, cell, offset, vx, vy, vz, ids=None, on_device=False):
    if on_device:
        n = int(cell.numel())
        args = [_ptr(cell), _ptr(offset), _ptr(vx), _ptr(vy), _ptr(vz), _ptr(ids)]
    else:
        arrs = [np.ascontiguousarray(cell, dtype=np.int32), np.ascontiguousarray(offset, dtype=np.float32),
                np.ascontiguousarray(vx, dtype=np.float32), np.ascontiguousarray(vy, dtype=np.float32),
                np.ascontiguousarray(vz, dtype=np.float32)]
        idsa = None if ids is None else np.ascontiguousarray(ids, dtype=np.uint32)
        n = arrs[0].size
        args = [a.ctypes.data for a in arrs] + [None if idsa is None else idsa.ctypes.data]
    check(lib.pic_load_particles(h, species, n, *args, int(bool(on_device))))


def load_particles_si(h, species, x_m, v_m_per_s, ids=None, on_device=False):
    """pic_load_particles_si: positions (m) and an n x 3 velocity array (m/s), FP64."""
    if on_device:
        n = int(x_m.numel())
        args = [_ptr(x_m), _ptr(v_m_per_s), _ptr(ids)]
    else:
        x = np.ascontiguousarray(x_m, dtype=np.float64)
        v = np.ascontiguousarray(v_m_per_s, dtype=np.float64).reshape(-1, 3)
        if v.shape[0] != x.size:
            raise ValueError("v_m_per_s must be n x 3")
        idsa = None if ids is None else np.ascontiguousarray(ids, dtype=np.uint32)
        n = x.size
        args = [x.ctypes.data, v.ctypes.data, None if idsa is None else idsa.ctypes.data]
    check(lib.pic_load_particles_si(h, species, n, *args, int(bool(on_device))))


def load_profile(h, species, n, density, temp_ev, drift=(0.0, 0.0, 0.0), id_base=0):
    d = np.ascontiguousarray(density, dtype=np.float64)
    t = np.ascontiguousarray(temp_ev, dtype=np.float64)
    dr = np.ascontiguousarray(drift, dtype=np.float64)
    dp_ = C.POINTER(C.c_double)
    check(lib.pic_load_profile(h, species, int(n), d.ctypes.data_as(dp_), t.ctypes.data_as(dp_),
                               dr.ctypes.data_as(dp_), int(id_base) & 0xFFFFFFFF))


def step(h, n_steps=1):
    check(lib.pic_step(h, int(n_steps)))


def sync(h):
    check(lib.pic_sync(h))


def count(h):
    out = (C.c_int64 * 2)()
    check(lib.pic_count(h, out))
    return int(out[0]), int(out[1])


def read_particles(h, species, max_n=None) -> dict:
    n_alive = count(h)[species]
    max_n = n_alive if max_n is None else max_n
    out = {"cell": np.zeros(max_n, np.int32), "off": np.zeros(max_n, np.float32), "vx": np.zeros(max_n, np.float32),
           "vy": np.zeros(max_n, np.float32), "vz": np.zeros(max_n, np.float32), "id": np.zeros(max_n, np.uint32)}
    n = C.c_int64()
    check(lib.pic_read_particles(h, species, max_n, C.byref(n), out["cell"].ctypes.data, out["off"].ctypes.data,
                                 out["vx"].ctypes.data, out["vy"].ctypes.data, out["vz"].ctypes.data,
                                 out["id"].ctypes.data))
    return {k: v[: n.value] for k, v in out.items()}


def read_field(h, n_nodes, n_species):
    phi = np.zeros(n_nodes)
    E = np.zeros(n_nodes)
    R = np.zeros(n_species * n_nodes, dtype=np.int64)
    check(lib.pic_read_field(h, phi.ctypes.data, E.ctypes.data, R.ctypes.data))
    return phi, E, R.reshape(n_species, n_nodes)


def read_moments(h, n_nodes, n_species, reset=False, field_energy_cap=0) -> dict:
    m = Moments()
    m.struct_size = C.sizeof(Moments)
    bufs = {"dens_sum": np.zeros(n_species * n_nodes), "phi_sum": np.zeros(n_nodes),
            "en_sum": np.zeros(n_species * n_nodes), "dens_diag_sum": np.zeros(n_species * n_nodes),
            "eepf": np.zeros(EEPF_BINS), "field_energy": np.zeros(max(1, field_energy_cap)),
            "ifedf": np.zeros(2 * IFEDF_BINS)}
    for k, v in bufs.items():
        setattr(m, k, v.ctypes.data)
    m.field_energy_cap = field_energy_cap
    m.reset = int(bool(reset))
    check(lib.pic_read_moments(h, C.byref(m)))
    out = {k: v for k, v in bufs.items()}
    for k in ("dens_sum", "en_sum", "dens_diag_sum"):
        out[k] = out[k].reshape(n_species, n_nodes)
    out["ifedf"] = out["ifedf"].reshape(2, IFEDF_BINS)
    out["electrode_charge"] = m.electrode_charge
    out["renewed"] = np.array(list(m.renewed))
    out["field_energy"] = out["field_energy"][: m.field_energy_n]
    out.update(step=m.step, n_steps=m.n_steps, n_diag=m.n_diag, n_alive=tuple(m.n_alive),
               absorbed=np.array([[m.absorbed[s][w] for w in range(2)] for s in range(2)]),
               see_emitted=m.see_emitted, ionizations=m.ionizations, candidates=np.array(list(m.candidates)),
               collisions=np.array([[m.collisions[s][k] for k in range(MAX_PROC)] for s in range(2)]),
               ke_sum=np.array(list(m.ke_sum)), pw_sum=np.array(list(m.pw_sum)), sort_interval=m.sort_interval)
    return out


def read_tuning(h) -> dict:
    t = Tuning()
    t.struct_size = C.sizeof(Tuning)
    check(lib.pic_read_tuning(h, C.byref(t)))
    return dict(tuned=bool(t.tuned), sort_interval=tuple(t.sort_interval), threads=tuple(t.threads),
                stages=tuple(t.stages), grid=tuple(t.grid),
                shape_ms=[list(t.shape_ms[s]) for s in range(2)], sort_ms=tuple(t.sort_ms),
                slope_ms=tuple(t.slope_ms))


def profile(h, enable=True):
    check(lib.pic_profile(h, int(bool(enable))))


def profile_read(h) -> dict:
    arr = (KernelStat * 8)()
    n = C.c_int()
    check(lib.pic_profile_read(h, arr, 8, C.byref(n)))
    return {arr[i].name.decode(): dict(launches=arr[i].launches, timed=arr[i].timed, total_ms=arr[i].total_ms)
            for i in range(n.value)}


def destroy(h):
    check(lib.pic_destroy(h))


def philox(seed: int, ctr_dev, out_dev, n: int, stream=None):
    check(lib.pic_philox(int(seed) & 0xFFFFFFFFFFFFFFFF, int(n), _ptr(ctr_dev), _ptr(out_dev), stream))


def deposit(n_cells, periodic, cell_dev, off_dev, R_dev, stream=None):
    check(lib.pic_deposit(int(n_cells), int(periodic), int(cell_dev.numel()), _ptr(cell_dev), _ptr(off_dev),
                          _ptr(R_dev), stream))


def sort_by_cell(n_cells, src: dict, dst: dict, n_live_dev=None, stream=None):
    """Counting sort of device SoA particles (dicts of torch tensors) by cell."""
    keys = ("cell", "off", "vx", "vy", "vz", "id")
    check(lib.pic_sort_by_cell(int(n_cells), int(src["cell"].numel()), *[_ptr(src[k]) for k in keys],
                               *[_ptr(dst[k]) for k in keys], _ptr(n_live_dev), stream))


def sort_by_cell_noalloc(n_cells, src: dict, dst: dict, n_live_dev=None, stream=None):
    """The same sort with the library's fixed scratch array (no device allocation)."""
    keys = ("cell", "off", "vx", "vy", "vz", "id")
    check(lib.pic_sort_by_cell_noalloc(int(n_cells), int(src["cell"].numel()), *[_ptr(src[k]) for k in keys],
                                       *[_ptr(dst[k]) for k in keys], _ptr(n_live_dev), stream))


def _f32(a):
    a = np.ascontiguousarray(a, dtype=np.float32)
    return a, a.ctypes.data_as(C.POINTER(C.c_float))


class MLP:
    """The warm-start network (``pic_mlp_*``): 3 layers, BF16 tensor-core products."""

    def __init__(self, n_in, n_hidden, n_out, seed=0):
        h = C.c_void_p()
        check(lib.pic_mlp_create(n_in, n_hidden, n_out, int(seed), C.byref(h)))
        self.h = h.value
        self.n_in, self.n_hidden, self.n_out = n_in, n_hidden, n_out

    def set_normalization(self, in_lo, in_hi, out_mean, out_sd):
        arrs = [_f32(a) for a in (in_lo, in_hi, out_mean, out_sd)]
        check(lib.pic_mlp_set_normalization(self.h, *[p for _, p in arrs]))

    def params(self):
        out = np.zeros(int(lib.pic_mlp_param_count(self.h)), np.float32)
        check(lib.pic_mlp_get_params(self.h, out.ctypes.data_as(C.POINTER(C.c_float))))
        return out

    def set_params(self, p):
        a, ptr = _f32(p)
        check(lib.pic_mlp_set_params(self.h, ptr))

    def gradients(self, X, Y):
        X, px = _f32(X); Y, py = _f32(Y)
        g = np.zeros(int(lib.pic_mlp_param_count(self.h)), np.float32)
        loss = C.c_float()
        check(lib.pic_mlp_gradients(self.h, px, py, X.shape[0], g.ctypes.data_as(C.POINTER(C.c_float)), C.byref(loss)))
        return float(loss.value), g

    def train(self, X, Y, epochs, lr=1e-3, record=True):
        X, px = _f32(X); Y, py = _f32(Y)
        curve = np.zeros(epochs, np.float32)
        check(lib.pic_mlp_train(self.h, px, py, X.shape[0], int(epochs), float(lr),
                                curve.ctypes.data_as(C.POINTER(C.c_float)) if record else None))
        return curve

    def adam_step(self, grads, lr):
        g, pg = _f32(grads)
        check(lib.pic_mlp_adam_step(self.h, pg, float(lr)))

    def warmstart_train(self, params, ne, ni, te, in_lo, in_hi, epochs, lr=1e-3, record=True):
        """pic_warmstart_train: params (cases x n_in), profiles (cases x points)."""
        d = lambda a: np.ascontiguousarray(a, dtype=np.float64)
        P, NE, NI, TE, LO, HI = (d(a) for a in (params, ne, ni, te, in_lo, in_hi))
        dp_ = C.POINTER(C.c_double)
        curve = np.zeros(max(int(epochs), 1), np.float32)
        check(lib.pic_warmstart_train(self.h, P.ctypes.data_as(dp_), NE.ctypes.data_as(dp_), NI.ctypes.data_as(dp_),
                                      TE.ctypes.data_as(dp_), P.shape[0], P.shape[1], NE.shape[1],
                                      LO.ctypes.data_as(dp_), HI.ctypes.data_as(dp_), int(epochs), float(lr),
                                      curve.ctypes.data_as(C.POINTER(C.c_float)) if record else None))
        return curve[: int(epochs)]

    def predict(self, X):
        X, px = _f32(X)
        Y = np.zeros((X.shape[0], self.n_out), np.float32)
        check(lib.pic_mlp_predict(self.h, px, X.shape[0], Y.ctypes.data_as(C.POINTER(C.c_float))))
        return Y

    def close(self):
        if getattr(self, "h", None):
            check(lib.pic_mlp_destroy(self.h))
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def gemm_bf16(A, ar, ac, B, br, bc, Cm, ldc, M, N, K, stream=None):
    check(lib.pic_gemm_bf16(_ptr(A), ar, ac, _ptr(B), br, bc, _ptr(Cm), ldc, M, N, K, stream))


class Batch:
    """Many independent cases stepped together (``pic_batch_*``).  ``cases[i]``
    is a borrowed :class:`Case` view for per-case loads and reads."""

    def __init__(self, cfgs, *, stream=None, sort_interval=0, capacities=None):
        descs = (CaseDesc * len(cfgs))()
        for i, cfg in enumerate(cfgs):
            cap = capacities[i] if capacities is not None else (0, 0)
            descs[i] = make_desc(cfg, stream=stream, capacity=cap, sort_interval=sort_interval)
        h = C.c_void_p()
        check(lib.pic_batch_create(descs, len(cfgs), C.byref(h)))
        self.h = h.value
        self.cases = []
        for i, cfg in enumerate(cfgs):
            v = Case.__new__(Case)
            v._view(cfg, lib.pic_batch_case(self.h, i))
            for t in cfg.get("xsec", []):
                if t["species"] < v.n_species:
                    load_xsec_table(v.h, t["species"], t["kind"], t["threshold"], t["energy"], t["sigma"])
            self.cases.append(v)

    def step(self, n=1):
        check(lib.pic_batch_step(self.h, int(n)))

    def sync(self):
        check(lib.pic_batch_sync(self.h))

    def launches(self):
        return int(lib.pic_batch_launches(self.h))

    def set_stages(self, stages):
        check(lib.pic_batch_set_stages(self.h, int(stages)))

    def set_shape(self, shape):
        check(lib.pic_batch_set_shape(self.h, int(shape)))

    def set_own_threshold(self, particles):
        check(lib.pic_batch_set_own_threshold(self.h, int(particles)))

    def tuning(self):
        """Launch shape, sort interval, whether the autotuner ran, and its timings."""
        sh, k, tu, sm = C.c_int(), C.c_int(), C.c_int(), C.c_float()
        ms, st = (C.c_float * 6)(), (C.c_float * 32)()
        check(lib.pic_batch_tuning(self.h, C.byref(sh), C.byref(k), C.byref(tu), ms, C.byref(sm), st))
        return dict(shape=sh.value, sort_interval=k.value, tuned=bool(tu.value), shape_ms=list(ms),
                    sort_ms=sm.value, step_ms=list(st))

    def retune(self):
        check(lib.pic_batch_retune(self.h))

    def freeze(self, i, frozen=True):
        check(lib.pic_batch_freeze(self.h, int(i), int(bool(frozen))))

    def replan(self):
        """Re-split the work items from the current particle counts before the next step."""
        lib.pic_batch_case(self.h, 0)

    def close(self):
        if getattr(self, "h", None):
            check(lib.pic_batch_destroy(self.h))
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Case:
    """A case on the current CUDA device: ``Case(cfg, parts)`` creates it, loads
    its tables and particles; ``step(n)``; ``particles(sp)``; ``moments()``."""

    def __init__(self, cfg: dict, parts=None, *, stream=None, allocator=None, capacity=(0, 0),
                 sort_interval=0, field_history=0):
        self.cfg = cfg
        self.n_cells = int(cfg["n_cells"])
        self.periodic = bool(cfg["periodic"])
        self.n_nodes = self.n_cells if self.periodic else self.n_cells + 1
        self.n_species = len(cfg["species"])
        self._desc = make_desc(cfg, stream=stream, allocator=allocator, capacity=capacity,
                               sort_interval=sort_interval, field_history=field_history)
        self._allocator = allocator
        self.h = create_case(self._desc)
        for t in cfg.get("xsec", []):
            if t["species"] < self.n_species:
                load_xsec_table(self.h, t["species"], t["kind"], t["threshold"], t["energy"], t["sigma"])
        if parts is not None:
            for s, p in enumerate(parts):
                self.load(s, p)

    def _view(self, cfg, handle):
        """Borrowed handle of a case owned by a batch (never destroyed here)."""
        self.cfg = cfg
        self.n_cells = int(cfg["n_cells"])
        self.periodic = bool(cfg["periodic"])
        self.n_nodes = self.n_cells if self.periodic else self.n_cells + 1
        self.n_species = len(cfg["species"])
        self.h = handle
        self._borrowed = True

    def load_profile(self, sp, n, density, temp_ev, drift=(0.0, 0.0, 0.0), id_base=0):
        load_profile(self.h, sp, n, density, temp_ev, drift, id_base)

    def warmstart_load(self, mlp, params, n_points, ion_temp_ev, id_base=0, max_per_species=0):
        prm = np.ascontiguousarray(params, dtype=np.float64)
        check(lib.pic_warmstart_load(self.h, mlp.h, prm.ctypes.data_as(C.POINTER(C.c_double)), prm.size,
                                     int(n_points), float(ion_temp_ev), int(id_base), int(max_per_species)))

    def load(self, sp, p, on_device=False):
        load_particles(self.h, sp, p["cell"], p["off"], p["vx"], p["vy"], p["vz"], p.get("id"), on_device)

    def load_si(self, sp, x_m, v_m_per_s, ids=None, on_device=False):
        load_particles_si(self.h, sp, x_m, v_m_per_s, ids, on_device)

    def clear_error(self):
        check(lib.pic_clear_error(self.h))

    def set_wait_limit(self, polls):
        check(lib.pic_set_wait_limit(self.h, int(polls)))

    def step(self, n=1):
        step(self.h, n)

    def sync(self):
        sync(self.h)

    def count(self):
        return count(self.h)

    def particles(self, sp):
        return read_particles(self.h, sp)

    def field(self):
        return read_field(self.h, self.n_nodes, self.n_species)

    def moments(self, reset=False, field_energy_cap=0):
        return read_moments(self.h, self.n_nodes, self.n_species, reset=reset, field_energy_cap=field_energy_cap)

    def clock(self, sp):
        """Collision clock 2 k + c of the live particles, in the order of ``particles``."""
        n = int(self.count()[sp])
        out = np.zeros(n, np.uint32)
        k = C.c_int64()
        check(lib.pic_read_clock(self.h, sp, n, C.byref(k), out.ctypes.data))
        return out[: k.value]

    def axial(self, sp):
        """Axial excursion z (m) of the live particles, in the order of ``particles``."""
        n = int(self.count()[sp])
        z = np.zeros(n, np.float32)
        k = C.c_int64()
        check(lib.pic_read_axial(self.h, sp, n, C.byref(k), z.ctypes.data))
        return z[: k.value]

    def tuning(self):
        return read_tuning(self.h)

    def set_step_shape(self, species, threads, stages):
        check(lib.pic_set_step_shape(self.h, species, threads, stages))

    def checkpoint(self) -> bytes:
        """The case's state between steps (pic_checkpoint_save) as bytes."""
        n = C.c_uint64()
        check(lib.pic_checkpoint_size(self.h, C.byref(n)))
        buf = C.create_string_buffer(n.value)
        check(lib.pic_checkpoint_save(self.h, buf, n.value))
        return buf.raw

    def restore(self, data: bytes):
        """Continue from a checkpoint taken from a case of the same descriptor."""
        buf = C.create_string_buffer(data, len(data))
        check(lib.pic_checkpoint_load(self.h, buf, len(data)))

    def profile(self, enable=True):
        profile(self.h, enable)

    def profile_read(self):
        return profile_read(self.h)

    def close(self):
        if getattr(self, "h", None) and not getattr(self, "_borrowed", False):
            destroy(self.h)
        self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
