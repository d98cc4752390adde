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


def _stable_cases(collapse=0):
    """Four small rising bubbles of different sizes and parameters that stay
    finite for thousands of steps (density ratios 50 to 100, constant mobility)."""
    out = []
    for i, (nx, ny) in enumerate([(40, 72), (64, 48), (70, 50), (33, 45)]):
        p, _ = inputs.small_case(mobility=0, density_ratio=50.0 + 15 * i)
        p = dict(p, nx=nx, ny=ny, pl_n=0.6 + 0.1 * i, collapse_h=collapse)
        R = min(nx, ny) / 5.0
        C = inputs.round_to_fp32(inputs.bubble_fields(nx, ny, 2, p["xi"], [(nx / 2, ny / 3, R, 3)], seed=i,
                                                      noise=1e-8))
        out.append((p, C))
    return out


@pytest.mark.parametrize("collapse", [0, 1])
def test_persistent_launch_equals_per_step_launches(lbm, collapse):
    """One cooperative launch per 4096 steps (the first replayed from its
    graph, the rest a direct launch) gives the per-step launches' values bit
    for bit: same items, same per-node arithmetic."""
    cases = _stable_cases(collapse)
    per_step = lbm.Batch([p for p, _ in cases])
    persistent = lbm.Batch([p for p, _ in cases])
    persistent.set_persistent(True)
    for i, (_, C) in enumerate(cases):
        per_step.case(i).set_fields(C)
        persistent.case(i).set_fields(C)
    per_step.step(4096 + 37)
    persistent.step(4096 + 37)
    names = ("C1", "p", "ux", "uy", "tau", "g") + (() if collapse else ("h",))
    for i in range(len(cases)):
        assert persistent.case(i).observables()["step"] == 4096 + 37
        for n in names:
            assert np.array_equal(persistent.case(i).field(n), per_step.case(i).field(n)), (i, n)


def test_persistent_barrier_wait_limit_returns_timeout(lbm):
    """A grid-barrier wait limited to one poll gives up (the CTAs finish their
    items microseconds apart): the call returns LBM_E_TIMEOUT without a fault
    or a hang, the cases must be set again, and after that the same batch
    steps normally and matches a single lattice."""
    cases = []
    for i in range(8):
        p, b = inputs.sweep_case(192, density_ratio=100.0)
        cases.append((p, inputs.round_to_fp32(inputs.bubble_fields(p["nx"], p["ny"], 2, p["xi"], b, seed=i,
                                                                   noise=1e-8))))
    batch = lbm.Batch([p for p, _ in cases])
    batch.set_persistent(True, spin_limit=1)
    for i, (_, C) in enumerate(cases):
        batch.case(i).set_fields(C)
    with pytest.raises(lbm.LbmError) as ei:
        batch.step(6)
    assert ei.value.status == -5
    with pytest.raises(lbm.LbmError) as ei:   # the stopped launch left no whole step
        batch.step(2)
    assert ei.value.status == -6
    batch.set_persistent(True)              # the default limit
    for i, (_, C) in enumerate(cases):
        batch.case(i).set_fields(C)
    batch.step(6)
    ref = lbm.Lattice(cases[3][0])
    ref.set_fields(cases[3][1])
    ref.step(6)
    for n in ("C1", "p", "uy", "tau", "g", "h"):
        assert np.array_equal(batch.case(3).field(n), ref.field(n)), n


def test_persistent_batch_matches_oracle(lbm):
    """Two cases of one persistent batch against the FP64 oracle directly, per
    field within max(1e-5, 4 x the FP32-build deviation) after 300 steps."""
    import oracle

    def rel(a, b):
        return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-12 * b.size))

    cases = _stable_cases()[:2]
    batch = lbm.Batch([p for p, _ in cases])
    batch.set_persistent(True)
    for i, (_, C) in enumerate(cases):
        batch.case(i).set_fields(C)
    batch.step(300)
    for i, (p, C) in enumerate(cases):
        o64, o32 = oracle.Oracle(p), oracle.Oracle(p, "f32")
        for o in (o64, o32):
            o.set_fields(C)
            o.step(300)
        for n in ("C1", "p", "ux", "uy", "tau", "g", "h"):
            ref = o64.field(n)
            err, floor = rel(batch.case(i).field(n), ref), rel(o32.field(n), ref)
            assert err <= max(1e-5, 4.0 * floor), (i, n, err, floor)


def test_batch_run_to_terminal_matches_a_per_case_loop(lbm):
    """lbm_batch_run (the terminal criterion and the window-averaged rise
    velocity inside the library) against the same criterion written here
    around single lattices stepped window by window."""
    window, rtol, max_steps = 500, 0.02, 6000
    cases = []
    for i, (nx, ny) in enumerate([(48, 96), (40, 80), (56, 96)]):
        p, _ = inputs.small_case(mobility=0, density_ratio=20.0 + 10 * i)
        p = dict(p, nx=nx, ny=ny, pl_n=0.7 + 0.1 * i)
        C = inputs.round_to_fp32(inputs.bubble_fields(nx, ny, 2, p["xi"], [(nx / 2, ny / 3, nx / 6, 3)], seed=i,
                                                      noise=1e-8))
        cases.append((p, C))
    batch = lbm.Batch([p for p, _ in cases])
    batch.set_persistent(True)
    for i, (_, C) in enumerate(cases):
        batch.case(i).set_fields(C)
    res = batch.run(window=window, rtol=rtol, max_steps=max_steps, top_margin=1.5)
    for i, (p, C) in enumerate(cases):
        lat = lbm.Lattice(p)
        lat.set_fields(C)
        ob = lat.observables()
        ys, top, steps = [ob["centroid"][1]], p["ny"] - 1 - 1.5 * ob["d_eq"], 0
        while True:
            lat.step(window)
            steps += window
            ob = lat.observables()
            ys.append(ob["centroid"][1])
            u = np.diff(ys) / window
            if len(u) >= 3 and all(abs(u[-j] - u[-j - 1]) < rtol * abs(u[-j]) for j in (1, 2)):
                outcome = "terminal"
            elif ys[-1] > top:
                outcome = "top"
            elif steps >= max_steps:
                outcome = "max_steps"
            else:
                continue
            break
        assert res[i]["outcome"] == outcome and res[i]["steps_run"] == steps, (i, res[i]["outcome"], outcome)
        assert res[i]["rise_velocity"] == float(u[-1])
        raw = np.array(ob["raw"])
        raw[10] = u[-1] * raw[6]
        assert res[i]["drag_coefficient"] == lbm.lbm_postprocess(p, raw)["drag_coefficient"]


def test_fp16_batch_equals_fp16_single_lattices(lbm):
    """FP16 storage of g (with the C state) in a persistent batch: the same
    values as each case stepped alone in that form."""
    cases = [(dict(p, collapse_h=1, storage=1), C) for p, C in _stable_cases()]
    batch = lbm.Batch([p for p, _ in cases])
    batch.set_persistent(True)
    singles = []
    for i, (p, C) in enumerate(cases):
        batch.case(i).set_fields(C)
        lat = lbm.Lattice(p)
        lat.set_fields(C)
        singles.append(lat)
    batch.step(123)
    for lat in singles:
        lat.step(123)
    for i, lat in enumerate(singles):
        for n in ("C1", "p", "ux", "uy", "tau", "g"):
            assert np.array_equal(batch.case(i).field(n), lat.field(n)), (i, n)


def test_batch_run_reports_diverged_and_step_limit_cases(lbm):
    """A case that diverges (the R = 10 bubble at density ratio 1000) is an
    outcome of lbm_batch_run, not an error: it stops as 'diverged' within its
    first windows while the others run on, to the step limit here."""
    p_bad, b_bad = inputs.small_case(density_ratio=1000.0)
    p_ok, b_ok = inputs.small_case(density_ratio=20.0)
    cases = [(p_ok, b_ok), (p_bad, b_bad), (dict(p_ok, pl_n=0.9), b_ok)]
    batch = lbm.Batch([p for p, _ in cases])
    batch.set_persistent(True)
    for i, (p, b) in enumerate(cases):
        batch.case(i).set_fields(inputs.bubble_fields(p["nx"], p["ny"], 2, p["xi"], b, seed=i, noise=1e-8))
    res = batch.run(window=200, rtol=1e-9, max_steps=1000, top_margin=0.0)
    assert res[1]["outcome"] == "diverged" and res[1]["steps_run"] <= 400
    for i in (0, 2):
        assert res[i]["outcome"] in ("max_steps", "top") and res[i]["steps_run"] <= 1000
        assert np.isfinite(res[i]["rise_velocity"]) and np.isfinite(res[i]["drag_coefficient"])
