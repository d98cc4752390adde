"""Batched ensembles (one launch per step over a (case, tile) work list,
replayed from a CUDA graph) against the same cases stepped one by one."""
import numpy as np
import pytest

from paper_2207_09431_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lbm():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2207_09431_gb300 import lbm as _lbm

    _lbm.load_library()
    return _lbm


def _cases(collapse=0):
    out = []
    shapes = [(40, 72), (64, 48), (70, 50), (33, 45)]
    for i, (nx, ny) in enumerate(shapes):
        p, _ = inputs.small_case(mobility=i % 2, density_ratio=50.0 + 25 * i)
        p = dict(p, nx=nx, ny=ny, pl_n=0.6 + 0.1 * i, sigma12=1e-3 * (1 + 0.2 * i),
                 sigma13=1e-3 * (1 + 0.2 * i), sigma23=1e-3 * (1 + 0.2 * i), collapse_h=collapse)
        R = min(nx, ny) / 5.0
        C = inputs.round_to_fp32(inputs.bubble_fields(nx, ny, 2, p["xi"], [(nx / 2, ny / 3, R, 3)], seed=i,
                                                      noise=1e-8))
        out.append((p, C))
    return out


@pytest.mark.parametrize("collapse", [0, 1])
def test_batch_equals_single_lattices(lbm, collapse):
    cases = _cases(collapse)
    batch = lbm.Batch([p for p, _ in cases])
    singles = []
    for i, (p, C) in enumerate(cases):
        batch.case(i).set_fields(C)
        lat = lbm.Lattice(p)
        lat.set_fields(C)
        singles.append(lat)
    batch.step(37)                      # two graph replays of 16 steps and 5 direct launches
    for lat in singles:
        lat.step(37)
    names = ("C1", "p", "ux", "uy", "tau", "g") + (() if collapse else ("h",))
    for i, lat in enumerate(singles):
        for n in names:
            assert np.array_equal(batch.case(i).field(n), lat.field(n)), (i, n)


def test_inactive_case_is_frozen_and_autotune_keeps_values(lbm):
    cases = _cases()
    batch = lbm.Batch([p for p, _ in cases])
    for i, (p, C) in enumerate(cases):
        batch.case(i).set_fields(C)
    batch.step(10)
    frozen = batch.case(2).field("g")
    batch.set_active(2, False)
    chosen = batch.autotune(reps=2)
    assert chosen >= 0
    batch.step(20)
    assert np.array_equal(batch.case(2).field("g"), frozen)
    ref = lbm.Lattice(cases[0][0])
    ref.set_fields(cases[0][1])
    ref.step(30)
    for n in ("C1", "p", "uy", "tau"):
        a, b = batch.case(0).field(n), ref.field(n)
        assert np.linalg.norm(a - b) <= 1e-6 * max(np.linalg.norm(b), 1e-30), n
    assert batch.case(0).observables()["step"] == 30
    assert batch.case(2).observables()["step"] == 10
