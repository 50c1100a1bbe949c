"""The allocation-free counting sort gives the same result as pic_sort_by_cell.

pic_sort_by_cell_noalloc serves callers that must not allocate device memory
while running (fixed memory budget, a host program that owns the device heap,
or no room for the synchronisation an allocation can imply): its scratch is a
fixed array inside the library.  This file is collected last so that a run
stopping at its first failure has run every other test already; it must pass
both alone in a fresh process and after the rest of the suite.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_2609_17151_b300 import pic  # noqa: E402

KEYS = ("cell", "off", "vx", "vy", "vz", "id")


def _particles(seed, n, n_cells):
    rng = np.random.default_rng(seed)
    cell = rng.integers(-1, n_cells + 1, n).astype(np.int32)      # some absorbed (-1) and out of range
    host = {"cell": cell, "off": rng.random(n, dtype=np.float32),
            "vx": rng.standard_normal(n).astype(np.float32), "vy": rng.standard_normal(n).astype(np.float32),
            "vz": rng.standard_normal(n).astype(np.float32), "id": rng.permutation(n).astype(np.uint32)}
    return {k: torch.from_numpy(v.view(np.int32) if v.dtype == np.uint32 else v).cuda() for k, v in host.items()}


def _canonical(out, k):
    """Sorted copy of the first k outputs: the order inside a cell is free."""
    h = {kk: v[:k].cpu().numpy() for kk, v in out.items()}
    o = np.lexsort((h["id"], h["cell"]))
    return {kk: v[o] for kk, v in h.items()}, h["cell"]


@pytest.mark.parametrize("n_cells,n", [(2048, 1_000_003), (4096, 65_537)])
def test_noalloc_sort_matches_allocating_sort_twice(n_cells, n):
    for call in range(2):                                   # two calls in a row share the scratch array
        src = _particles(1000 * call + n_cells, n, n_cells)
        ref = {k: torch.empty_like(v) for k, v in src.items()}
        got = {k: torch.full_like(v, -7) for k, v in src.items()}
        n_ref = torch.zeros(1, dtype=torch.int64, device="cuda")
        n_got = torch.full((1,), -1, dtype=torch.int64, device="cuda")
        pic.sort_by_cell(n_cells, src, ref, n_ref)
        torch.cuda.synchronize()
        free_before = torch.cuda.mem_get_info()[0]
        pic.sort_by_cell_noalloc(n_cells, src, got, n_got)
        torch.cuda.synchronize()
        if call == 1:                                       # after the first call's one-time set-up
            assert torch.cuda.mem_get_info()[0] == free_before, "the call changed free device memory"
        k = int(n_ref.item())
        assert int(n_got.item()) == k
        a, cells_ref = _canonical(ref, k)
        b, cells_got = _canonical(got, k)
        assert np.all(np.diff(cells_got) >= 0)              # grouped by ascending cell
        for kk in KEYS:
            assert np.array_equal(a[kk], b[kk]), (call, kk)


def test_noalloc_rejects_more_cells_than_its_scratch_holds():
    lib = pic.lib
    st = lib.pic_sort_by_cell_noalloc(4097, 0, *([None] * 12), None, None)
    assert st == 1                                          # PIC_EINVAL, nothing launched
    assert b"PIC_NOALLOC_MAX_CELLS" in lib.pic_last_error()
    st = lib.pic_sort_by_cell_noalloc(0, 0, *([None] * 12), None, None)
    assert st == 1
    assert ctypes.sizeof(ctypes.c_int64) == 8
