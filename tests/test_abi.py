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
    """The ctypes mirror of pic_case_desc / pic_moments has the C sizes."""
    import paper_2609_17151_b300.pic as pic
    src = open(os.path.join(ROOT, "include", "pic1d3v.h")).read()
    assert "PIC_DESC_VERSION 1u" in src
    # 8-byte aligned structs with the documented field counts
    assert ctypes.sizeof(pic.CaseDesc) % 8 == 0
    assert ctypes.sizeof(pic.Moments) % 8 == 0
    assert [f[0] for f in pic.CaseDesc._fields_][:4] == ["struct_size", "version", "periodic", "n_cells"]
