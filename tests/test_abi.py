"""The C-ABI library loads and exports every entry point include/biotmg.h declares (CPU:
only host-side layout helpers are called; nothing touches a GPU)."""
import ctypes
import os
import re

import numpy as np

import synthetic

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "biotmg.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(bmg_[a-z0-9_]+)\s*\(", src)))


def test_header_declares_the_paper_calls():
    syms = declared_symbols()
    for name in ("bmg_assemble", "bmg_setup_hierarchy", "bmg_vcycle", "bmg_fgmres_solve",
                 "bmg_apply", "bmg_residual"):
        assert name in syms


def test_library_exports_every_declared_symbol():
    import paper_2107_04060_gb300 as bmg
    lib = ctypes.CDLL(bmg.LIB_PATH)
    missing = [s for s in declared_symbols() if not hasattr(lib, s)]
    assert not missing, missing


def test_layout_helpers():
    import paper_2107_04060_gb300 as bmg
    for n in (1, 2, 7, 8, 16, 511, 512, 2048):
        P = bmg.pitch(n)
        assert P >= n + 1 and P % 8 == 0 and P - (n + 1) < 8
        assert bmg.block_len(n) == (n + 1) * P
        assert bmg.vector_len(n) == 10 * (n + 1) * P
        masks = synthetic.dirichlet_masks(n)
        free = sum(int((~m).sum()) for m in masks.values())
        assert bmg.free_dofs(n) == free
    assert bmg.free_dofs(512) == 2619394 and bmg.free_dofs(16) == 2498


def test_pack_roundtrip():
    import paper_2107_04060_gb300 as bmg
    n = 5
    f = synthetic.uniform_field(n, 4)
    x = bmg.pack(n, f)
    g = bmg.unpack(n, x)
    for t in synthetic.TYPES:
        assert np.array_equal(f[t], g[t])
    # unused slots are zero
    assert np.count_nonzero(x) == sum(int(np.count_nonzero(v)) for v in f.values())
