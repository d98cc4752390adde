"""The stability comparison of the two directional-derivative schemes (Sec.
2.2, reading R2) runs through the C ABI on the paper-size rising bubble at
density ratio 1000 and reports per case the steps survived, the Mach number
and the share of liquid nodes at a tau clamp."""
import pytest

pytestmark = pytest.mark.gpu


def test_survival_table_on_a_corner_of_the_grid():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2207_09431_gb300 import inputs, stability

    rows = []
    for fd in (0, 1):
        cases = inputs.paper_grid_cases(fd_scheme=fd, ns=(0.5, 1.0), eotvos=(10.0,), log10_mo=(-1.0,))
        rows += stability.survival(cases, steps=2000, chunk=500)
    assert len(rows) == 4
    for r in rows:
        assert set(r) >= {"n", "Eo", "log10_Mo", "fd_scheme", "steps", "diverged", "mach", "tau_clamped"}
        assert r["steps"] == 2000 or r["diverged"]
        assert 0.0 <= r["tau_clamped"] <= 1.0
    print("stability:", rows)
