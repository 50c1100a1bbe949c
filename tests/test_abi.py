"""The C-ABI library builds, loads without a GPU and exports every entry
point that include/*.h declares (no compute calls here)."""
import ctypes
import glob
import os
import re

from paper_2609_17151_b300 import build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        names.update(re.findall(r"\b(pic_[a-z0-9_]+)\s*\(", src))
    return names


def test_library_builds_and_exports_every_declared_symbol():
    path = build.build()
    lib = ctypes.CDLL(path)
    names = declared_symbols()
    assert {"pic_create_case", "pic_load_xsec_table", "pic_load_particles", "pic_step", "pic_read_moments",
            "pic_destroy"} <= names
    for n in sorted(names):
        assert hasattr(lib, n), n


def test_status_strings_and_null_handling_without_gpu():
    lib = ctypes.CDLL(build.build())
    lib.pic_status_str.restype = ctypes.c_char_p
    assert lib.pic_status_str(0) == b"ok"
    assert lib.pic_status_str(4) == b"particle capacity exceeded"
    lib.pic_create_case.argtypes = [ctypes.c_void_p, ctypes.c_void_p]
    assert lib.pic_create_case(None, None) == 1          # PIC_EINVAL, no device touched
    lib.pic_destroy.argtypes = [ctypes.c_void_p]
    assert lib.pic_destroy(None) == 0


def test_descriptor_layout_matches_header():
    """The ctypes mirrors of pic_case_desc, pic_moments and pic_tuning have the
    sizes and field offsets the C compiler gives the header's structs."""
    import subprocess
    import tempfile
    import paper_2609_17151_b300.pic as pic
    src = open(os.path.join(ROOT, "include", "pic1d3v.h")).read()
    assert f"PIC_DESC_VERSION {pic.DESC_VERSION}u" in src
    mirrors = {"pic_case_desc": pic.CaseDesc, "pic_moments": pic.Moments, "pic_tuning": pic.Tuning}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "pic1d3v.h"', "int main(void) {"]
    for cname, py in mirrors.items():
        lines.append(f'printf("{cname} size %zu\\n", sizeof({cname}));')
        for f in py._fields_:
            lines.append(f'printf("{cname} {f[0]} %zu\\n", offsetof({cname}, {f[0]}));')
    lines.append("return 0; }")
    with tempfile.TemporaryDirectory() as d:
        c_file, exe = os.path.join(d, "layout.c"), os.path.join(d, "layout")
        open(c_file, "w").write("\n".join(lines))
        subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), c_file, "-o", exe])
        out = subprocess.check_output([exe], text=True).split("\n")
    got = {tuple(ln.split()[:2]): int(ln.split()[2]) for ln in out if ln.strip()}
    for cname, py in mirrors.items():
        assert got[(cname, "size")] == ctypes.sizeof(py), cname
        for f in py._fields_:
            assert got[(cname, f[0])] == getattr(py, f[0]).offset, (cname, f[0])


def test_non_finite_descriptor_is_rejected_before_any_device_work():
    """Every floating-point quantity of the descriptor must be finite: a NaN or
    an infinity is PIC_EINVAL from pic_create_case, checked before the call
    touches a device (so this runs without a GPU)."""
    import math

    from paper_2609_17151_b300 import pic
    from paper_2609_17151_b300 import workloads as W
    cfg, _ = W.ccp_case(seed=1, n_cells=32, gap=32 * 5e-5, n_per_species=10)
    bad = [("B", (0.0, math.nan, 0.0)), ("bg_charge", math.inf), ("see_gamma", math.nan),
           ("harmonics", [(13.56e6, math.inf, 0.0)]), ("E_ext", (0.0, 0.0, -math.inf))]
    for key, val in bad:
        c = dict(cfg)
        c[key] = val
        d = pic.make_desc(c)
        h = ctypes.c_void_p()
        assert pic.lib.pic_create_case(ctypes.byref(d), ctypes.byref(h)) == 1, key
        assert b"not finite" in pic.lib.pic_last_error(), key
        assert not h.value
