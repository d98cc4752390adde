"""The surrogate pipeline end to end: terminal states of 1024 seeded 100 x 200
rising-bubble cases from the batched solver, an ensemble of five networks
trained on them by the library's kernels, and 128 held-out cases solved in
full as the yardstick.  Shows what the network gains over the solver alone (time
to an answer) and at what error, and that the solver answers every case the
network does not trust."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def trained():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2207_09431_gb300 import surrogate

    stream = torch.cuda.Stream()
    summary, model = surrogate.evaluate(n_train=1024, n_test=128, stream=stream, return_model=True)
    print("surrogate:", summary)
    return summary, model, stream


def test_trusted_drag_coefficients_within_5_percent(trained):
    """Every trusted answer within 5 % of the solver's C_D.  Trust needs the
    members' agreement and a small local out-of-fold residual: agreement alone
    leaves misses of up to 16 %, where the labels themselves scatter (they are
    terminal states under a stopping rule)."""
    s, _, _ = trained
    assert s["train_converged"] >= 256
    assert s["trusted"] >= 8
    assert s["judged"] >= 6
    assert s["cd_within_5pct"] == 1.0
    assert s["cd_rel_err_max"] < 0.05
    assert s["cd_within_5pct_spread_only"] <= s["cd_within_5pct"]


def test_network_answers_much_faster_than_the_solver(trained):
    s, _, _ = trained
    assert s["speedup_trusted"] >= 100.0


def test_solver_fallback_outside_the_training_box(trained):
    """A case beyond the sampled Eotvos range is not trusted and is answered
    by the solver, with the same result as solving it directly."""
    from paper_2207_09431_gb300 import inputs, surrogate

    _, model, stream = trained
    base = inputs.ensemble_cases(1, seed=4242, grids=((100, 200),))[0]
    p, b, meta = base
    far = (p, b, dict(meta, Eo=250.0))          # features only: outside the box
    U, CD, used_solver, _ = model.answer([far], stream=stream, max_steps=4000)
    assert used_solver.tolist() == [True]
    direct, _ = surrogate.run_to_terminal([far], stream=stream, max_steps=4000)
    # same case, same kernel body (the autotuner may pick another tile shape)
    np.testing.assert_allclose([U[0], CD[0]], [direct[0]["U_t"], direct[0]["C_D"]], rtol=1e-6)
