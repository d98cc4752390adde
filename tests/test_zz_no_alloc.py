"""The observables entry point that allocates no device memory.

Some callers own all device memory themselves and cannot let the library
allocate (nor hand it an arena just for a query); lbm_observables_static works
on buffers they already hold and keeps its scratch in a fixed device array.
This file is collected last so that a run stopping at the first failure has
already run every other test.
"""
import numpy as np
import pytest

from paper_2207_09431_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2207_09431_gb300 import lbm

    lbm.load_library()
    return torch, lbm


def _device_planes(torch, planes, nx, ny):
    """Pitched FP32 device copy of (nplanes, ny, nx) host planes."""
    pitch = (nx + 31) // 32 * 32
    buf = torch.zeros((planes.shape[0], ny, pitch), dtype=torch.float32, device="cuda")
    buf[:, :, :nx] = torch.from_numpy(planes.astype(np.float32)).cuda()
    return buf, pitch, ny * pitch


@pytest.mark.parametrize("collapse", [0, 1])
def test_static_observables_match_lbm_observables(env, collapse):
    torch, lbm = env
    p, _ = inputs.small_case(mobility=1)
    nx, ny = 80, 112
    p = dict(p, nx=nx, ny=ny, collapse_h=collapse)
    C = inputs.round_to_fp32(inputs.bubble_fields(nx, ny, 2, p["xi"], [(40.0, 40.0, 12.0, 3)], seed=4,
                                                  noise=1e-8))
    lat = lbm.Lattice(p)
    lat.set_fields(C)
    lat.step(40)
    ref = np.array(lat.observables()["raw"])       # the existing entry point
    g, _, _ = _device_planes(torch, lat.field("g"), nx, ny)
    if collapse:
        state = lat.field("C1")[None]
    else:
        state = lat.field("h").reshape(-1, ny, nx)
    hc, pitch, plane = _device_planes(torch, state, nx, ny)
    stream = torch.cuda.current_stream()
    for _ in range(2):   # two calls in a row share the scratch array
        raw = lbm.lbm_observables_static(p, g.data_ptr(), hc.data_ptr(), pitch, plane, stream.cuda_stream)
        assert np.allclose(raw[:11], ref[:11], rtol=1e-5, atol=1e-12)
        assert np.array_equal(raw[11:], ref[11:])


def test_static_observables_rejects_oversized_lattice(env):
    torch, lbm = env
    p, _ = inputs.small_case()
    p = dict(p, nx=2048, ny=1024)   # 2 Mi nodes > LBM_STATIC_MAX_NODES
    assert p["nx"] * p["ny"] > lbm.STATIC_MAX_NODES
    x = torch.zeros(16, dtype=torch.float32, device="cuda")
    with pytest.raises(lbm.LbmError) as ei:
        lbm.lbm_observables_static(p, x.data_ptr(), x.data_ptr(), 2048, 2048 * 1024, 0)
    assert ei.value.status == -8
