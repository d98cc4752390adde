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


def _case(kind):
    """(params, initial C, inflow ux or None) of one lattice form."""
    if kind == "walls":
        p, _ = inputs.small_case(mobility=1)
        nx, ny = 80, 112
        p = dict(p, nx=nx, ny=ny)
        C = inputs.bubble_fields(nx, ny, 2, p["xi"], [(40.0, 40.0, 12.0, 3)], seed=4, noise=1e-8)
        return p, C, None
    if kind == "three_periodic":
        p, discs = inputs.three_comp_case(nx=72, mobility=1, seed=2)
        C = inputs.bubble_fields(72, 72, 3, p["xi"], discs, seed=5, noise=1e-8, periodic_y=True)
        return p, C, None
    # open x: velocity inlet and convective outlet, a gas bubble across the
    # inlet so that the mirrored inlet columns enter every sum
    p, _, ux = inputs.open_channel_case(0.7, ny=48, nx=64, u_in=0.02)
    p = dict(p, rho=(1.0, 1.0, 0.1), tau=(0.8, 0.8, 0.5), sigma12=1e-3, sigma13=1e-3, sigma23=1e-3, xi=4.0,
             D0=4.0 / 300.0, gravity=1e-6, gas_comp=3)
    C = inputs.bubble_fields(64, 48, 2, 4.0, [(5.0, 24.0, 9.0, 3)], seed=6, noise=1e-8)
    return p, C, ux


@pytest.mark.parametrize("kind,collapse", [("walls", 0), ("walls", 1), ("three_periodic", 0),
                                           ("three_periodic", 1), ("open_x", 0)])
def test_static_observables_match_lbm_observables(env, kind, collapse):
    torch, lbm = env
    p, C, ux = _case(kind)
    p = dict(p, collapse_h=collapse)
    nx, ny, nh = p["nx"], p["ny"], p["ncomp"] - 1
    lat = lbm.Lattice(p)
    lat.set_fields(inputs.round_to_fp32(C), ux=ux)
    lat.step(40)
    ref = np.array(lat.observables()["raw"])       # the existing entry point
    g, _, _ = _device_planes(torch, lat.field("g"), nx, ny)
    if collapse:
        state = np.stack([lat.field("C1")] + ([lat.field("C2")] if nh == 2 else []))
    else:
        state = lat.field("h").reshape(-1, ny, nx)
    hc, pitch, plane = _device_planes(torch, state, nx, ny)
    stream = torch.cuda.current_stream()
    for _ in range(2):   # two calls in a row share the scratch array
        raw = lbm.lbm_observables_static(p, g.data_ptr(), hc.data_ptr(), pitch, plane, stream.cuda_stream)
        assert np.allclose(raw[:11], ref[:11], rtol=1e-5, atol=1e-9), (kind, raw[:11] - ref[:11])
        assert np.array_equal(raw[11:], ref[11:])


def test_static_observables_rejects_fp16_storage_and_capture(env):
    torch, lbm = env
    p, _ = inputs.small_case()
    nx, ny = p["nx"], p["ny"]
    x = torch.zeros(9 * ny * nx, dtype=torch.float32, device="cuda")
    with pytest.raises(lbm.LbmError) as ei:   # this call reads FP32 populations only
        lbm.lbm_observables_static(dict(p, collapse_h=1, storage=1), x.data_ptr(), x.data_ptr(), nx, nx * ny, 0)
    assert ei.value.status == -1
    s = torch.cuda.Stream()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=s):
        try:
            lbm.lbm_observables_static(p, x.data_ptr(), x.data_ptr(), nx, nx * ny, s.cuda_stream)
            refused = None
        except lbm.LbmError as e:
            refused = e.status
    assert refused == -1


def test_static_observables_rejects_oversized_lattice(env):
    torch, lbm = env
    p, _ = inputs.small_case()
    p = dict(p, nx=2048, ny=1024)   # 2 Mi nodes > LBM_STATIC_MAX_NODES
    assert p["nx"] * p["ny"] > lbm.STATIC_MAX_NODES
    x = torch.zeros(16, dtype=torch.float32, device="cuda")
    with pytest.raises(lbm.LbmError) as ei:
        lbm.lbm_observables_static(p, x.data_ptr(), x.data_ptr(), 2048, 2048 * 1024, 0)
    assert ei.value.status == -8
