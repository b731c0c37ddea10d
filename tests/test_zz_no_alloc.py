"""The allocation-free totals entry point against the workspace-based one.

Callers that cannot allocate device memory (code running during CUDA graph capture, hosts
that hand the library a fixed pool) use eslbm_read_totals_noalloc on a state buffer they
already hold.  Its scratch is a device array inside the library, so the first call on a
device does the set-up; this file is collected last and must pass on its own too.
"""
import numpy as np
import pytest

from paper_2403_13406_gb300 import eslbm, inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

CASES = [
    (dict(dim=1, system="sw", nx=1000, V=4.0, g=9.81), "fp64", lambda: inputs.sw_random_1d(1000, seed=3)),
    (dict(dim=1, system="sw", nx=4099, V=4.0, g=9.81), "fp32", lambda: inputs.sw_random_1d(4099, seed=8)),
    (dict(dim=2, system="burgers", nx=37, ny=29, V=3.0), "fp32",
     lambda: inputs.burgers_2d(37, 29, seed=5, noise=1e-3)),
]


def physical_from_logical(f, cfg, s):
    """Planes p with T(s) p = f: population k is rolled back by sign_k * s along its axis."""
    out = np.empty_like(f)
    q = 2 if cfg.dim == 1 else 4
    M = f.shape[0] // q
    for k in range(q):
        axis = 0 if cfg.dim == 1 else (k & 1)
        sign = (1 if k == 0 else -1) if cfg.dim == 1 else (1 if k < 2 else -1)
        ax = f.ndim - 1 - axis  # numpy axis of x (last) or y
        for m in range(M):
            out[k * M + m] = np.roll(f[k * M + m], -sign * s, axis=ax - 1)
    return out


@pytest.mark.parametrize("kw,precision,init", CASES)
def test_noalloc_totals_match(kw, precision, init):
    cfg = eslbm.make_config(precision=precision, omega_mode="entropic", **kw)
    sim = eslbm.Simulation(cfg)
    sim.init_equilibrium(init())
    sim.step(2)
    ref = sim.totals()
    f_logical = sim.distributions(host=True)
    sim.close()
    dtype = torch.float64 if precision == "fp64" else torch.float32
    stream = torch.cuda.current_stream()
    for pending in (0, 3, -5):
        phys = torch.from_numpy(physical_from_logical(f_logical, cfg, pending)).to(dtype).cuda()
        # two calls in a row: the shared scratch keeps the previous call's contents
        host = np.empty_like(ref)
        eslbm.read_totals_noalloc(cfg, phys.data_ptr(), pending, host.ctypes.data, 0, stream.cuda_stream)
        dev = torch.empty(len(ref), dtype=torch.float64, device="cuda")
        eslbm.read_totals_noalloc(cfg, phys.data_ptr(), pending, dev.data_ptr(), 1, stream.cuda_stream)
        torch.cuda.synchronize()
        np.testing.assert_allclose(host, ref, rtol=1e-12, atol=1e-12)
        np.testing.assert_allclose(dev.cpu().numpy(), ref, rtol=1e-12, atol=1e-12)


def test_noalloc_rejects_bad_arguments():
    cfg = eslbm.make_config(1, "burgers", 64, V=1.5)
    buf = torch.zeros(2 * 64, dtype=torch.float32, device="cuda")
    out = np.empty(3)
    with pytest.raises(eslbm.EslbmError) as e:
        eslbm.read_totals_noalloc(cfg, 0, 0, out.ctypes.data, 0, None)
    assert e.value.status == eslbm.ERR_ARG
    with pytest.raises(eslbm.EslbmError) as e:
        eslbm.read_totals_noalloc(cfg, buf.data_ptr() + 4, 0, out.ctypes.data, 0, None)
    assert e.value.status == eslbm.ERR_ARG
    bad = eslbm.make_config(1, "burgers", 0, V=1.5)
    with pytest.raises(eslbm.EslbmError) as e:
        eslbm.read_totals_noalloc(bad, buf.data_ptr(), 0, out.ctypes.data, 0, None)
    assert e.value.status == eslbm.ERR_ARG


def test_noalloc_totals_in_a_captured_graph():
    """The reason the call exists: totals recorded inside a CUDA graph capture (where no memory can
    be allocated) and replayed.  The set-up call comes first, outside the capture; during capture a
    host output is refused (it would need a stream synchronization) and leaves the capture intact."""
    cfg = eslbm.make_config(1, "sw", 2048, V=4.0, g=9.81, precision="fp32", omega_mode="entropic")
    sim = eslbm.Simulation(cfg)
    sim.init_equilibrium(inputs.sw_random_1d(2048, seed=11))
    sim.step(1)
    ref = sim.totals()
    f_logical = sim.distributions(host=True)
    sim.close()
    phys = torch.from_numpy(physical_from_logical(f_logical, cfg, 0)).to(torch.float32).cuda()
    out = torch.zeros(len(ref), dtype=torch.float64, device="cuda")
    side = torch.cuda.Stream()
    with torch.cuda.stream(side):
        eslbm.read_totals_noalloc(cfg, phys.data_ptr(), 0, out.data_ptr(), 1, side.cuda_stream)  # set-up
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    host = np.empty_like(ref)
    with torch.cuda.graph(graph):
        st = torch.cuda.current_stream().cuda_stream
        with pytest.raises(eslbm.EslbmError) as e:
            eslbm.read_totals_noalloc(cfg, phys.data_ptr(), 0, host.ctypes.data, 0, st)
        assert e.value.status == eslbm.ERR_ARG
        eslbm.read_totals_noalloc(cfg, phys.data_ptr(), 0, out.data_ptr(), 1, st)
    for _ in range(2):  # two replays in a row on the shared scratch
        out.zero_()
        graph.replay()
        torch.cuda.synchronize()
        np.testing.assert_allclose(out.cpu().numpy(), ref, rtol=1e-12, atol=1e-12)
    # the graph reads the buffer at replay time: new contents, new totals
    phys.mul_(0.5)
    graph.replay()
    torch.cuda.synchronize()
    assert abs(out[2].item() - 0.5 * ref[2]) <= 1e-9 * abs(ref[2])
