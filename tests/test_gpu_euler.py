"""2D Euler on the GPU path (FP64, omega = 2, scheme I): the isentropic vortex (strength 5,
background rho = p = 1, velocity (1, 1), on [0, 10]^2) is advected without change of shape, so the
exact solution at time t is the initial field translated by t (1, 1).  The paper prints no Euler
values; this pins the Euler equilibrium and the composite step by the exact solution: the error falls
at the scheme's order under refinement, and mass, momentum and energy are conserved."""
import math

import numpy as np
import pytest

from paper_2403_13406_gb300 import eslbm, inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)


def vortex_error(N):
    V = 8.0
    cfg = eslbm.make_config(2, "euler", N, N, V=V, gamma=1.4, precision="fp64", omega=2.0, scheme="I")
    sim = eslbm.Simulation(cfg)
    u0 = inputs.euler_vortex_2d(N, N)
    sim.init_equilibrium(u0)
    dt = 24 * (10.0 / N) / V
    n = N // 32  # t = n dt = 0.9375 on every grid
    sim.step(n)
    u = sim.moments(host=True)
    tot = sim.totals()
    sim.close()
    t = n * dt
    ex = inputs.euler_vortex_2d(N, N, centre=(5 + t, 5 + t))
    dx2 = (10.0 / N) ** 2
    for m in range(4):  # conserved totals (cell sums)
        assert abs(tot[2 + m] - u0[m].sum()) <= 1e-12 * abs(u0[m]).sum()
    return math.sqrt(dx2 * float(np.sum((u[0] - ex[0]) ** 2)))


def test_euler_vortex_converges_at_fourth_order():
    errs = [vortex_error(N) for N in (128, 256, 512)]
    orders = [math.log2(a / b) for a, b in zip(errs, errs[1:])]
    assert errs[-1] < 1e-5
    assert orders[-1] > 3.5, (errs, orders)
