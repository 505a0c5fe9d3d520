"""The C-ABI library builds, loads and exports every symbol the header declares."""
import ctypes
import os
import re

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "celeste.h")).read()
    return sorted(set(re.findall(r"^(?:int|int64_t)\s+(celeste_\w+)\(", src, re.M)))


def test_library_exports_every_declared_symbol():
    import __graft_entry__
    __graft_entry__.build()
    from paper_1803_00113_gb300 import build_lib, celeste
    lib = ctypes.CDLL(build_lib.LIB)
    declared = _declared()
    assert declared, "no declarations found"
    for name in declared:
        assert hasattr(lib, name), name
    assert sorted(celeste.exported_symbols()) == sorted(declared)


def test_struct_layouts_match_header():
    from paper_1803_00113_gb300 import celeste
    assert celeste.IMAGE_DTYPE.itemsize == 256
    assert celeste.PATCH_DTYPE.itemsize == 32
    assert ctypes.sizeof(celeste._Tuning) == 32
    assert ctypes.sizeof(celeste._Model) == 4 * 4 + 8 * (32 + 1 + 4 + 16 + 64 + 256 + 6)


def test_colouring_is_proper_and_greedy():
    import __graft_entry__
    __graft_entry__.build()
    from paper_1803_00113_gb300 import celeste
    import fields
    p = fields.batched(seed=2, n_sources=60, max_images_per_band=1)
    col = celeste.color_sources(p.nbr_ptr, p.nbr_idx)
    for s in range(p.n_sources):
        nb = p.nbr_idx[p.nbr_ptr[s]:p.nbr_ptr[s + 1]]
        assert np.all(col[nb] != col[s])
        lower = {int(col[t]) for t in nb if t < s}
        assert int(col[s]) == min(set(range(len(lower) + 1)) - lower)


def test_colouring_equals_the_oracle_classes():
    """The library's host colouring and the oracle's colour classes follow the
    same greedy rule (ascending id) and must agree exactly."""
    import __graft_entry__
    __graft_entry__.build()
    from paper_1803_00113_gb300 import celeste
    import fields
    from oracle import newton as ON
    for seed in (3, 4):
        p = fields.batched(seed=seed, n_sources=80, max_images_per_band=1, max_neighbours=8)
        col = celeste.color_sources(p.nbr_ptr, p.nbr_idx)
        classes = ON.overlap_classes(p)
        assert len(classes) == int(col.max()) + 1
        for c, members in enumerate(classes):
            assert members == [int(s) for s in np.flatnonzero(col == c)]
