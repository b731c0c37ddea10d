"""The paper's printed error tables reproduced by the sm_103a path (FP64, through the C ABI).

The oracle is pinned to the first rows of these tables (tests/test_oracle_tables.py); the GPU
reaches every row, down to the finest grids, with the same conventions: cells at x_j = j dx,
dx = 1/N, data at equilibrium, n = floor(T / dt) steps with dt = 24 dx / V in double precision,
errors at t = n dt.  Printed values have four significant digits.
"""
import math

import numpy as np
import pytest

import oracle as O
from _golden import table
from paper_2403_13406_gb300 import eslbm, inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)


def burgers_exact(x, t):
    """Pre-shock solution of u_t + (u^2/2)_x = 0 for u0 = sin 2 pi x, by characteristics."""
    xi = x.copy()
    for _ in range(60):
        xi = xi - (xi + np.sin(2 * np.pi * xi) * t - x) / (1 + 2 * np.pi * np.cos(2 * np.pi * xi) * t)
    return np.sin(2 * np.pi * xi)


def l2(e, dx):
    return math.sqrt(dx * float(np.sum(e * e)))


def n_steps(T, N, V, step=24):
    return int(math.floor(T / (step * (1.0 / N) / V)))


def run(system, N, V, u0, n, scheme="I", mode="fixed", f0=None, **kw):
    cfg = eslbm.make_config(1, system, N, V=V, precision="fp64", omega_mode=mode, scheme=scheme, **kw)
    sim = eslbm.Simulation(cfg)
    if f0 is None:
        sim.init_equilibrium(u0)
    else:
        sim.init_distributions(f0)
    sim.step(n)
    u = sim.moments(host=True)
    diag = sim.diagnostics()
    sim.close()
    return u, diag


def burgers_grids():
    """Grids of Tables 1, 4 and 5: the dx column, printed to four digits, does not fix N (1/dx =
    3275.5 and 8382.2 in rows 5 and 7); N_{i+1} = floor(1.6 N_i) from N = 500 reproduces every
    printed dx, and it is the reading used here."""
    Ns = [500]
    while len(Ns) < 8:
        Ns.append(int(math.floor(1.6 * Ns[-1])))
    for N, row in zip(Ns, table("table1_burgers_order.txt")):
        assert float("%.3E" % (1.0 / N)) == row[0]
    return Ns


def burgers_error(N, scheme="I", mode="fixed", theta=None, V=1.2, T=0.1):
    u0 = inputs.sine_1d(N)
    f0 = None if theta is None else np.concatenate([theta * u0, (1 - theta) * u0])
    n = n_steps(T, N, V)
    u, diag = run("burgers", N, V, u0, n, scheme=scheme, mode=mode, f0=f0)
    assert diag["fallbacks"] == 0
    return l2(u[0] - burgers_exact(inputs.grid_1d(N), n * 24 * (1.0 / N) / V), 1.0 / N)


@pytest.mark.parametrize("row", range(8))
def test_table1_burgers(row):
    """Table 1: second-order scheme R T (own step dx/V) and the fourth-order composite scheme."""
    dx, e2, e4 = table("table1_burgers_order.txt")[row]
    N = burgers_grids()[row]
    V, T = 1.2, 0.1
    assert abs(burgers_error(N) - e4) <= 1e-3 * e4
    n = n_steps(T, N, V, step=1)
    u, _ = run("burgers", N, V, inputs.sine_1d(N), n, scheme="plain")
    e = l2(u[0] - burgers_exact(inputs.grid_1d(N), n * (1.0 / N) / V), 1.0 / N)
    assert abs(e - e2) <= 1e-3 * e2


@pytest.mark.parametrize("row", range(8))
def test_table4_burgers_entropic(row):
    """Table 4: the entropic relaxation parameter keeps the fourth-order errors."""
    dx, e = table("table4_burgers_entropic.txt")[row]
    assert abs(burgers_error(burgers_grids()[row], mode="entropic") - e) <= 1e-3 * e


def test_table2_shallow_water():
    """Table 2: Err-Estim_h and Err-Estim_u (g = 1, V = 1.2, T = 5/16, h0 = 1/2 + 1/5 sin 2 pi x)."""
    V, g, T = 1.2, 1.0, 5.0 / 16.0
    sols = {}
    for k in range(7, 16):
        N = 1 << k
        n = n_steps(T, N, V)
        u, _ = run("sw", N, V, inputs.sw_sine_1d(N, h_mean=0.5, h_amp=0.2), n, g=g)
        sols[N] = (u[0], u[1] / u[0])
    for dx, eh, eu in table("table2_sw_order.txt"):
        N = int(round(1.0 / dx))
        (hc, uc), (hf, uf) = sols[N], sols[2 * N]
        assert abs(l2(hc - hf[::2], dx) - eh) <= 2e-4 * eh + 1e-15
        assert abs(l2(uc - uf[::2], dx) - eu) <= 2e-4 * eu + 1e-15


@pytest.mark.parametrize("tag,dx,e1,e2", [(r[0], r[1], r[2], r[3]) for r in table("table5_schemes_burgers.txt")])
def test_table5_schemes_i_ii(tag, dx, e1, e2):
    """Table 5, schemes (I) and (II) at equilibrium and off equilibrium (theta = 1/4)."""
    N = int(round(1.0 / dx))
    theta = None if tag == "eq" else 0.25
    assert abs(burgers_error(N, "I", theta=theta) - e1) <= 1e-3 * e1
    assert abs(burgers_error(N, "II", theta=theta) - e2) <= 1e-3 * e2


def test_table6_linear_sixth_order():
    """Table 6: |a| = sqrt(6)/12 V makes schemes (I) and (II) sixth order; every row."""
    V = 1.2
    a = math.sqrt(6) / 12 * V
    errs = []
    for dx, e1, e2, _e3, _e4 in table("table6_linear_transport.txt"):
        N = int(round(1.0 / dx))
        n = n_steps(10.0, N, V)
        t = n * 24 * (1.0 / N) / V
        exact = np.sin(2 * np.pi * (inputs.grid_1d(N) - a * t))
        for scheme, ref in (("I", e1), ("II", e2)):
            u, _ = run("linear", N, V, inputs.sine_1d(N), n, scheme=scheme, a=(a, 0.0))
            err = l2(u[0] - exact, 1.0 / N)
            assert abs(err - ref) <= 2e-3 * ref
        errs.append((dx, err))
    (d1, x1), (d2, x2) = errs[-2], errs[-1]
    assert math.log(x1 / x2) / math.log(d1 / d2) > 5.8


@pytest.mark.parametrize("precision", ["fp64"])
def test_fourth_order_2d_linear_gpu(precision):
    """D2Q4 linear transport on the GPU path converges at fourth order to u0(x - a t) up to 512^2
    (the staged 2D stage kernel: rows are multiples of 16 bytes)."""
    V, a = 1.0, (0.2, 0.1)
    errs = []
    for N in (64, 128, 256, 512):
        cfg = eslbm.make_config(2, "linear", N, N, V=V, a=a, precision=precision, omega=2.0)
        sim = eslbm.Simulation(cfg)
        sim.init_equilibrium(inputs.linear_sine_2d(N, N))
        n = N // 8
        sim.step(n)
        u = sim.moments(host=True)
        sim.close()
        t = n * 24 / N / V
        X, Y = inputs.grid_2d(N, N)
        ex = np.sin(2 * np.pi * (X - a[0] * t)) * np.cos(2 * np.pi * (Y - a[1] * t))
        errs.append(math.sqrt(float(np.mean((u[0] - ex) ** 2))))
    orders = [math.log2(errs[i] / errs[i + 1]) for i in range(3)]
    assert orders[-1] > 3.6 and sum(orders) / 3 > 3.5, (errs, orders)


def burgers_2d_solution(N, V, c, u0, n, precision="fp64"):
    cfg = eslbm.make_config(2, "burgers", N, N, V=V, c=c, precision=precision, omega_mode="entropic")
    sim = eslbm.Simulation(cfg)
    sim.init_equilibrium(u0)
    sim.step(n)
    u = sim.moments(host=True)[0]
    d = sim.diagnostics()
    sim.close()
    assert d["fallbacks"] == 0
    return u


def test_fourth_order_2d_entropic_burgers_gpu():
    """Entropic D2Q4 Burgers (flux c u^2 / 2, c = (1, 0.6)) on the GPU path: the oracle's result at
    64^2 to FP64 rounding, then fourth-order self-convergence at t = 1/8 (before the shock) up to 1024^2."""
    V, c = 6.0, (1.0, 0.6)

    def data(N):
        X, Y = inputs.grid_2d(N, N)
        return (0.5 + 0.25 * np.sin(2 * np.pi * X) * np.sin(2 * np.pi * Y))[None]

    m = O.Model(2, "burgers", 64, 64, V=V, c=c, omega_mode="entropic")
    f = O.init_equilibrium(m, data(64))
    O.composite_steps(m, f, 2)
    got = burgers_2d_solution(64, V, c, data(64), 2)
    ref = O.moments(m, f)[0]
    assert np.abs(got - ref).max() <= 1e-12 * np.abs(ref).max()
    sols = {N: burgers_2d_solution(N, V, c, data(N), N // 32) for N in (128, 256, 512, 1024)}
    d = [math.sqrt(float(np.mean((sols[N] - sols[2 * N][::2, ::2]) ** 2))) for N in (128, 256, 512)]
    orders = [math.log2(d[i] / d[i + 1]) for i in range(2)]
    assert min(orders) > 3.6, (d, orders)


def test_gaussian_2d_entropic_burgers_gpu():
    """The 2D Burgers data of Section 3.3 (u0 = exp(-100 |x - 1/2|^2), flux c u^2 / 2, c = (1, 0.6))
    with V = 3 to t = 1/16 on periodic grids of N = 2^k cells: self-convergence differences fall at
    fourth order once the Gaussian is resolved (orders above 3.5 from 512^2 to 4096^2)."""
    V, c = 3.0, (1.0, 0.6)
    sols = {N: burgers_2d_solution(N, V, c, inputs.gaussian_2d(N, N), N // 128) for N in (512, 1024, 2048, 4096)}
    d = [math.sqrt(float(np.mean((sols[N] - sols[2 * N][::2, ::2]) ** 2))) for N in (512, 1024, 2048)]
    orders = [math.log2(d[i] / d[i + 1]) for i in range(2)]
    assert min(orders) > 3.5, (d, orders)
