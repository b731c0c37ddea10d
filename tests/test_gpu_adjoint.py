"""Reverse mode through the C ABI: dot-product tests of the transposed linear map, central
finite differences of the GPU forward, and a CPU FP64 reference gradient (finite differences of
the oracle).  The adjoint is checked to 1e-6 relative."""
import numpy as np
import pytest

import oracle as O
from paper_2403_13406_gb300 import eslbm, inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2403_13406_gb300.autograd import evolve  # noqa: E402

CASES = {
    "burgers1d": (dict(dim=1, system="burgers", nx=48, V=1.5), lambda: inputs.random_scalar_1d(48, seed=2)),
    "sw1d": (dict(dim=1, system="sw", nx=40, V=4.0, g=9.81), lambda: inputs.sw_random_1d(40, seed=3, u_amp=0.2)),
    "burgers2d": (dict(dim=2, system="burgers", nx=14, ny=11, V=3.0, c=(1.0, 0.6)),
                  lambda: inputs.burgers_2d(14, 11, seed=5, noise=0.02)),
    # amplitude 0.03: every cell keeps its entropic root during the 3 steps (the default 0.05 on
    # this 12 x 10 grid sends 14 relaxations to the fallback omega = 1, where the forward map
    # is not differentiable and finite differences straddle the switch)
    "sw2d": (dict(dim=2, system="sw", nx=12, ny=10, V=8.0, g=9.81),
             lambda: inputs.sw_random_2d(12, 10, seed=6, h_amp=0.03, u_amp=0.03)),
    "euler": (dict(dim=2, system="euler", nx=12, ny=10, V=8.0, gamma=1.4),
              lambda: inputs.euler_vortex_2d(12, 10, length=4.0, centre=(2.0, 2.0), strength=2.0)),
}


def sim_for(kw, mode, precision="fp64", scheme="I"):
    return eslbm.Simulation(eslbm.make_config(precision=precision, omega_mode=mode, scheme=scheme, **kw))


def objective_grad(sim, u0, target, n, K):
    u = torch.from_numpy(u0).cuda().requires_grad_(True)
    uT = evolve(u, sim, n, K)
    J = 0.5 * ((uT - target) ** 2).sum()
    J.backward()
    return float(J.detach()), u.grad.cpu().numpy()


def forward_J(sim, u0, target, n):
    sim.init_equilibrium(u0)
    sim.step(n)
    uT = sim.moments(host=True)
    return 0.5 * float(((uT - target.cpu().numpy()) ** 2).sum())


@pytest.mark.parametrize("dim,scheme", [(1, "I"), (2, "I"), (1, "III"), (2, "IV")])
def test_dot_product_linear(dim, scheme):
    """<A x, y> = <x, A^T y> for the linear map u0 -> u_T of linear transport (omega = 2)."""
    if dim == 1:
        kw = dict(dim=1, system="linear", nx=53, V=1.0, a=(0.37, 0.0))
        shape = (1, 53)
    else:
        kw = dict(dim=2, system="linear", nx=13, ny=9, V=1.0, a=(0.2, -0.15))
        shape = (1, 9, 13)
    rng = np.random.default_rng(1)
    x, y = rng.standard_normal(shape), rng.standard_normal(shape)
    sim = sim_for(kw, "fixed", scheme=scheme)
    sim.init_equilibrium(x)
    sim.step(3)
    Ax = sim.moments(host=True)
    ATy = sim.gradient(torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda(), 3, K=2).cpu().numpy()
    lhs, rhs = float((Ax * y).sum()), float((x * ATy).sum())
    assert abs(lhs - rhs) <= 1e-12 * max(abs(lhs), 1.0)
    sim.close()


@pytest.mark.parametrize("name", list(CASES))
def test_gradient_matches_central_differences(name):
    kw, init = CASES[name]
    mode = "fixed" if name == "euler" else "entropic"
    sim = sim_for(kw, mode)
    u0 = init()
    rng = np.random.default_rng(7)
    target = torch.from_numpy(u0 * (1 + 0.01 * rng.standard_normal(u0.shape))).cuda()
    n = 3
    J, grad = objective_grad(sim, u0, target, n, K=2)
    flat = u0.reshape(-1)
    def J_at(idx, dx):
        x = u0.copy().reshape(-1)
        x[idx] += dx
        return forward_J(sim, x.reshape(u0.shape), target, n)

    for idx in rng.choice(flat.size, 6, replace=False):
        # fourth-order central difference: truncation O(h^4) ~ 1e-16 and rounding
        # ~ 2e-16 |J| / h ~ 1e-12 |J|; the second-order stencil at h = 1e-6 has a rounding
        # floor of 2e-10 |J|, which at |J| ~ 1 is above the 1e-6 relative bar
        h = 1e-4 * max(1.0, abs(flat[idx]))
        fd = (8.0 * (J_at(idx, h) - J_at(idx, -h)) - (J_at(idx, 2 * h) - J_at(idx, -2 * h))) / (12.0 * h)
        g = grad.reshape(-1)[idx]
        assert abs(g - fd) <= 1e-6 * max(abs(fd), np.abs(grad).max() * 1e-3), (idx, g, fd)
    sim.close()


def test_gradient_against_oracle_reference():
    """FP64 CPU reference gradient: central differences of the oracle's forward for every input."""
    kw, init = CASES["sw1d"]
    N = 16
    kw = dict(kw, nx=N)
    u0 = inputs.sw_random_1d(N, seed=3, u_amp=0.2)
    rng = np.random.default_rng(3)
    target = u0 * (1 + 0.01 * rng.standard_normal(u0.shape))
    n = 2
    m = O.Model(1, "sw", N, V=4.0, g=9.81, omega_mode="entropic")

    def J_oracle(u):
        f = O.init_equilibrium(m, u)
        O.composite_steps(m, f, n)
        return 0.5 * float(((O.moments(m, f) - target) ** 2).sum())

    ref = np.zeros_like(u0)
    for idx in np.ndindex(u0.shape):
        eps = 1e-6 * max(1.0, abs(u0[idx]))
        up, dn = u0.copy(), u0.copy()
        up[idx] += eps
        dn[idx] -= eps
        ref[idx] = (J_oracle(up) - J_oracle(dn)) / (2 * eps)
    sim = sim_for(kw, "entropic")
    _, grad = objective_grad(sim, u0, torch.from_numpy(target).cuda(), n, K=1)
    assert np.abs(grad - ref).max() <= 1e-6 * np.abs(ref).max()
    sim.close()


def test_checkpoint_interval_does_not_change_the_gradient():
    kw, init = CASES["sw1d"]
    sim = sim_for(kw, "entropic")
    u0 = init()
    y = torch.from_numpy(np.random.default_rng(2).standard_normal(u0.shape)).cuda()
    u = torch.from_numpy(u0).cuda()
    grads = [sim.gradient(u, y, 5, K=k).cpu().numpy() for k in (1, 2, 5, 7)]
    for g in grads[1:]:
        assert np.array_equal(g, grads[0])
    sim.close()


def test_fp32_adjoint_close_to_fp64():
    """The FP32 adjoint agrees with the FP64 one to ~1e-4 relative (measured 1.4e-4 here): the
    implicit derivative of the entropic omega divides by F'(t*) ~ |delta|^2, which amplifies the
    FP32 rounding of the state."""
    kw, init = CASES["sw1d"]
    u0 = init()
    y = torch.from_numpy(np.random.default_rng(4).standard_normal(u0.shape)).cuda()
    u = torch.from_numpy(u0).cuda()
    g = {}
    for prec in ("fp32", "fp64"):
        sim = sim_for(kw, "entropic", precision=prec)
        g[prec] = sim.gradient(u, y, 4, K=2).cpu().numpy()
        sim.close()
    assert np.linalg.norm(g["fp32"] - g["fp64"]) <= 1e-3 * np.linalg.norm(g["fp64"])
