"""Shifted storage: the state holds f - fbar for a reference equilibrium fbar = f^eq(u_ref).

The scheme is unchanged, so the parity bars against the FP64 oracle are those of the
plain storage (1e-12 relative max-norm in FP64, 1e-5 relative L2 in FP32); transport
is still a permutation of the stored values; the batched and the noalloc paths
agree with the single-lattice handle; and the FP32 rounding error of a long run is
smaller than with the plain storage.
"""
import numpy as np
import pytest

import oracle as O
from paper_2403_13406_gb300 import eslbm, inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

CASES = {
    # name: (dim, system, nx, ny, kwargs, initial data, u_ref)
    "burgers1d": (1, "burgers", 1000, 1, dict(V=1.5), lambda nx, ny: inputs.random_scalar_1d(nx, seed=2), (0.5,)),
    "linear1d": (1, "linear", 777, 1, dict(V=1.0, a=(0.37, 0.0)), lambda nx, ny: inputs.random_scalar_1d(nx, seed=4),
                 (0.0,)),
    "sw1d": (1, "sw", 1000, 1, dict(V=4.0, g=9.81), lambda nx, ny: inputs.sw_random_1d(nx, seed=3), (1.0, 0.0)),
    "burgers2d": (2, "burgers", 37, 29, dict(V=3.0, c=(1.0, 0.6)),
                  lambda nx, ny: inputs.burgers_2d(nx, ny, seed=5, noise=1e-3), (0.5,)),
    "sw2d": (2, "sw", 33, 27, dict(V=8.0, g=9.81), lambda nx, ny: inputs.sw_random_2d(nx, ny, seed=6),
             (1.0, 0.02, -0.01)),
}
EULER = (2, "euler", 40, 36, dict(V=8.0, gamma=1.4), lambda nx, ny: inputs.euler_vortex_2d(nx, ny),
         (1.0, 1.0, 1.0, 3.5))


def rel_max(a, b):
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


def rel_l2(a, b):
    return float(np.linalg.norm((a - b).ravel()) / max(np.linalg.norm(b.ravel()), 1e-300))


def run(case, mode, precision, nsteps, scheme="I", shifted=True):
    dim, system, nx, ny, kw, init, uref = case
    u0 = init(nx, ny)
    cfg = eslbm.make_config(dim, system, nx, ny, precision=precision, omega_mode=mode, scheme=scheme,
                            u_ref=uref if shifted else None, **kw)
    sim = eslbm.Simulation(cfg)
    sim.init_equilibrium(u0)
    sim.step(nsteps)
    f = sim.distributions(host=True)
    u = sim.moments(host=True)
    tot = sim.totals()
    diag = sim.diagnostics()
    sim.close()
    return u0, f, u, tot, diag


def oracle_run(case, mode, nsteps, scheme="I"):
    dim, system, nx, ny, kw, init, _ = case
    m = O.Model(dim, system, nx, ny, omega_mode=mode, **kw)
    f = O.init_equilibrium(m, init(nx, ny))
    O.composite_steps(m, f, nsteps, scheme=scheme)
    return m, f


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("mode", ["fixed", "entropic"])
def test_shifted_fp64_matches_oracle(name, mode):
    _, f, u, _, diag = run(CASES[name], mode, "fp64", 2)
    m, ref = oracle_run(CASES[name], mode, 2)
    assert rel_max(f, ref) <= 1e-12
    assert rel_max(u, O.moments(m, ref)) <= 1e-12


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("mode", ["fixed", "entropic"])
def test_shifted_fp32_matches_oracle(name, mode):
    _, f, _, _, _ = run(CASES[name], mode, "fp32", 2)
    _, ref = oracle_run(CASES[name], mode, 2)
    assert rel_l2(f, ref) <= 1e-5


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_shifted_euler_scheme_iii(precision):
    _, f, _, _, _ = run(EULER, "fixed", precision, 2, scheme="III")
    _, ref = oracle_run(EULER, "fixed", 2, scheme="III")
    if precision == "fp64":
        assert rel_max(f, ref) <= 1e-12
    else:
        assert rel_l2(f, ref) <= 1e-5


@pytest.mark.parametrize("name", ["sw1d", "sw2d"])
def test_shifted_totals_match_plain(name):
    """The totals (FP64 reductions of the reconstructed f) agree with those of the plain storage."""
    _, _, _, t1, _ = run(CASES[name], "entropic", "fp64", 2, shifted=True)
    _, _, _, t0, _ = run(CASES[name], "entropic", "fp64", 2, shifted=False)
    assert np.allclose(t1, t0, rtol=1e-12, atol=1e-12 * np.abs(t0).max())


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_shifted_transport_is_a_permutation(precision):
    dim, system, nx, ny, kw = 2, "sw", 67, 45, dict(V=10.0, g=9.81)
    cfg = eslbm.make_config(dim, system, nx, ny, precision=precision, u_ref=(1.0, 0.0, 0.0), **kw)
    sim = eslbm.Simulation(cfg)
    m = O.Model(dim, system, nx, ny, **kw)
    f0 = 1.0 + 0.1 * inputs.random_distributions(m.q * m.M, m.grid_shape, seed=11)
    sim.init_distributions(f0)
    before = sim.distributions(host=True)
    ref = before.copy()
    for s in (2, -4, 3):
        sim.transport(s)
        O.transport(m, ref, s)
    assert np.array_equal(sim.distributions(host=True), ref)
    sim.close()


def test_shifted_batch_matches_single():
    sizes = [(33, 27), (17, 40), (64, 9)]
    kw = dict(V=8.0, g=9.81)
    uref = (1.0, 0.0, 0.0)
    u0 = [inputs.sw_random_2d(nx, ny, seed=50 + i, h_amp=0.03, u_amp=0.03) for i, (nx, ny) in enumerate(sizes)]
    b = eslbm.Batch(eslbm.make_config(2, "sw", 1, 1, precision="fp32", omega_mode="fixed", u_ref=uref, **kw), sizes)
    b.init_equilibrium(u0)
    b.step(3)
    got = [u.cpu().numpy() for u in b.moments()]
    b.close()
    for (nx, ny), u, g in zip(sizes, u0, got):
        sim = eslbm.Simulation(eslbm.make_config(2, "sw", nx, ny, precision="fp32", omega_mode="fixed", u_ref=uref,
                                                 **kw))
        sim.init_equilibrium(u)
        sim.step(3)
        assert np.array_equal(g, sim.moments(host=True))
        sim.close()


def test_shifted_noalloc_totals():
    """eslbm_read_totals_noalloc on the raw buffer of a shifted state (right after the
    initialisation: first buffer, no pending shift) reproduces the handle's totals."""
    dim, system, nx, ny, kw, init, uref = CASES["sw1d"]
    cfg = eslbm.make_config(dim, system, nx, ny, precision="fp32", omega_mode="entropic", u_ref=uref, **kw)
    sim = eslbm.Simulation(cfg)
    sim.init_equilibrium(init(nx, ny))
    t_handle = sim.totals()
    out = np.empty(2 + sim.M)
    st = eslbm.lib().eslbm_read_totals_noalloc(eslbm.ctypes.byref(cfg), sim._fa.data_ptr(), 0, out.ctypes.data, 0,
                                               sim.stream.cuda_stream)
    assert st == eslbm.OK
    assert np.array_equal(out, t_handle)
    sim.close()


def test_shifted_reduces_fp32_rounding_error():
    """Long smooth 1D shallow-water run (h = 1 + 0.1 sin, 400 steps): the FP32 error against FP64 is
    several times smaller with the reference state (1, 0) than with the plain storage."""
    N, n = 4096, 400
    kw = dict(V=4.0, g=9.81)
    u0 = inputs.sw_sine_1d(N, 1.0, 0.1)
    out = {}
    for prec, uref in (("fp64", None), ("fp32", None), ("fp32s", (1.0, 0.0))):
        cfg = eslbm.make_config(1, "sw", N, precision=prec[:4], omega_mode="entropic", u_ref=uref, **kw)
        sim = eslbm.Simulation(cfg)
        sim.init_equilibrium(u0)
        sim.step(n)
        out[prec] = sim.moments(host=True)
        sim.close()
    e_plain = rel_l2(out["fp32"][0], out["fp64"][0])
    e_shift = rel_l2(out["fp32s"][0], out["fp64"][0])
    assert e_shift < e_plain / 3, (e_plain, e_shift)


def test_reference_outside_domain_is_rejected():
    cfg = eslbm.make_config(1, "sw", 64, V=4.0, g=9.81, u_ref=(-1.0, 0.0))
    with pytest.raises(eslbm.EslbmError) as e:
        eslbm.Simulation(cfg)
    assert e.value.status == eslbm.ERR_DOMAIN


@pytest.mark.parametrize("name", ["sw1d", "burgers2d"])
def test_shifted_gradient_matches_plain(name):
    """Reverse mode on the shifted storage: the same gradient as on the plain storage (FP64)."""
    dim, system, nx, ny, kw, init, uref = CASES[name]
    u0 = torch.as_tensor(init(nx, ny), device="cuda", dtype=torch.float64)
    lam = torch.as_tensor(np.random.default_rng(4).standard_normal(u0.shape), device="cuda")
    out = []
    for shifted in (False, True):
        cfg = eslbm.make_config(dim, system, nx, ny, precision="fp64", omega_mode="entropic",
                                u_ref=uref if shifted else None, **kw)
        sim = eslbm.Simulation(cfg)
        out.append(sim.gradient(u0, lam, n=3, K=2).cpu().numpy())
        sim.close()
    assert rel_max(out[1], out[0]) <= 1e-10
