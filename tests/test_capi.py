"""C-ABI library checks that need no GPU: it loads, exports every function that
include/lbm.h declares, validates parameters and post-processes observables
(host-only calls)."""
import math
import os
import re

import numpy as np
import pytest

import oracle
from oracle import observables as oobs
from paper_2207_09431_gb300 import inputs, lbm

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "lbm.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b((?:lbm|surr)_[a-z_]+)\s*\(", src)))


def test_library_exports_every_declared_symbol():
    lib = lbm.load_library()
    names = declared_functions()
    assert "lbm_step" in names and "lbm_create" in names
    for name in names:
        assert hasattr(lib, name), name
    assert sorted(lbm.EXPORTED) == names


def test_struct_sizes_match_header_layout():
    # lbm_params: 4 ints, 6 doubles, int, 4 doubles (n, k, tau_min, tau_max), 6 doubles, int,
    # 2 doubles, 3 ints -> with alignment padding
    import ctypes

    assert ctypes.sizeof(lbm.lbm_obs) == 8 * (1 + 3 + 3 + 1 + 2 + 2 + 1 + 1 + 1 + 1 + 1 + 3 + 15)
    assert lbm.lbm_version() >= 100


def test_required_bytes_and_validation():
    p, _ = inputs.small_case()
    nb = lbm.lbm_required_bytes(p)
    pitch = 64
    plane = 128 * pitch * 4
    # 18 g + 18 h + 2 tau + C + 3 mu + p, ux, uy, shear + SV planes, plus a small block
    assert nb >= (18 + 18 + 2 + 1 + 3 + 4 + 1) * plane
    bad = dict(p, ncomp=4)
    assert lbm.lbm_required_bytes(bad) == 0
    # degenerate and oversized lattices
    assert lbm.lbm_required_bytes(dict(p, nx=0)) == 0
    assert lbm.lbm_required_bytes(dict(p, ny=2)) == 0
    assert lbm.lbm_required_bytes(dict(p, nx=1, ny=3)) > 0
    assert lbm.lbm_required_bytes(dict(p, nx=65536, ny=65536)) == 0
    assert lbm.lbm_required_bytes(dict(p, sigma12=1e-3, sigma13=1e-3, sigma23=3e-3)) == 0
    assert lbm.lbm_required_bytes(dict(p, tau_min=2.0, tau_max=1.0)) == 0
    assert lbm.lbm_required_bytes(dict(p, storage=7)) == 0
    # FP16 storage of g rides on the collapsed form, in batches too
    assert lbm.lbm_required_bytes(dict(p, storage=1)) == 0
    q = dict(p, storage=1, collapse_h=1)
    assert lbm.lbm_required_bytes(q) == lbm.lbm_required_bytes(dict(q, storage=0)) > 0
    assert lbm.lbm_batch_required_bytes([q]) == lbm.lbm_batch_required_bytes([dict(q, storage=0)]) > 0
    # open x boundaries: population state only, at least 4 columns, not batched
    o = dict(p, open_x=1, u_in=0.02)
    assert lbm.lbm_required_bytes(o) > 0
    assert lbm.lbm_required_bytes(dict(o, collapse_h=1)) == 0
    assert lbm.lbm_required_bytes(dict(o, nx=3)) == 0
    assert lbm.lbm_batch_required_bytes([o]) == 0


def test_postprocess_matches_oracle_formulas():
    """The library's host post-processing (Eq. 37-40, 43-44) against the oracle's."""
    p, _ = inputs.small_case()
    rng = np.random.default_rng(3)
    raw = np.array([7000.0, 0.0, 1100.0, 6900.0, 0.0, 1000.0, 314.0, 314.0 * 31.7, 314.0 * 40.2,
                    314.0 * 1e-5, 314.0 * 2.3e-3, 22.0, 41.0, 30.0, 51.0]) * (1 + 0 * rng.random())
    got = lbm.lbm_postprocess(p, raw)
    want = oobs.postprocess(p, raw)
    for key in ("rise_velocity", "d_eq", "aspect_E", "drag_coefficient", "Re", "Eo", "Mo"):
        assert math.isclose(got[key], want[key], rel_tol=1e-12), key
    assert got["centroid"] == pytest.approx(want["centroid"], rel=1e-14)
    assert got["mass_thr"] == pytest.approx(want["mass_thr"], rel=1e-14)
