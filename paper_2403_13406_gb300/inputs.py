"""Seeded synthetic initial data shaped like the paper's test cases.

This module is shared by the CUDA path's tests, the bench and the oracle's
tests.  It holds initial conserved fields and workload parameters only: no
step of the lattice Boltzmann method is computed here.  It imports nothing
from the rest of the package.

Grid convention: periodic cells at x_j = j dx, dx = L / N (the convention
under which the oracle reproduces Table 2 digit for digit).  Fields are
float64 numpy arrays of shape (M, N) in 1D and (M, ny, nx) in 2D.
"""
import math

import numpy as np

SEED = 20240320


def grid_1d(n, length=1.0):
    return np.arange(n, dtype=np.float64) * (length / n)


def grid_2d(nx, ny, lx=1.0, ly=1.0):
    x = np.arange(nx, dtype=np.float64) * (lx / nx)
    y = np.arange(ny, dtype=np.float64) * (ly / ny)
    return np.meshgrid(x, y, indexing="xy")  # arrays of shape (ny, nx)


# ---- 1D scalar -------------------------------------------------------------

def sine_1d(n, mean=0.0, amp=1.0):
    """u0 = mean + amp sin(2 pi x) (Sections 3.1, 5.1, 6.2)."""
    x = grid_1d(n)
    return (mean + amp * np.sin(2.0 * np.pi * x))[None, :]


def random_scalar_1d(n, seed=SEED, mean=0.5, amp=0.25, modes=4):
    """Smooth random field: a few seeded Fourier modes about a mean."""
    rng = np.random.default_rng(seed)
    x = grid_1d(n)
    u = np.full(n, mean)
    c = rng.uniform(-1.0, 1.0, modes)
    c *= amp / np.abs(c).sum()
    ph = rng.uniform(0.0, 2.0 * np.pi, modes)
    for m in range(modes):
        u += c[m] * np.cos(2.0 * np.pi * (m + 1) * x + ph[m])
    return u[None, :]


# ---- 1D shallow water -------------------------------------------------------

def sw_sine_1d(n, h_mean=1.0, h_amp=0.1, u=0.0):
    """(h, hu) with h = h_mean + h_amp sin(2 pi x), uniform velocity u."""
    x = grid_1d(n)
    h = h_mean + h_amp * np.sin(2.0 * np.pi * x)
    return np.stack([h, h * u])


def sw_dam_break_1d(n, h_left=2.0, h_right=1.0, x0=0.5):
    """Dam break: h = h_left for x < x0, h_right otherwise, at rest (Section 5.2)."""
    x = grid_1d(n)
    h = np.where(x < x0, h_left, h_right).astype(np.float64)
    return np.stack([h, np.zeros(n)])


def sw_random_1d(n, seed=SEED, h_mean=1.0, h_amp=0.1, u_amp=0.1, modes=4):
    rng = np.random.default_rng(seed)
    x = grid_1d(n)
    h = np.full(n, h_mean)
    v = np.zeros(n)
    for m in range(modes):
        h += h_amp / modes * rng.uniform(-1, 1) * np.cos(2 * np.pi * (m + 1) * x + rng.uniform(0, 6.3))
        v += u_amp / modes * rng.uniform(-1, 1) * np.cos(2 * np.pi * (m + 1) * x + rng.uniform(0, 6.3))
    return np.stack([h, h * v])


# ---- 2D -----------------------------------------------------------------------

def burgers_2d(nx, ny, seed=SEED, noise=1e-3, mean=0.5, amp=0.25):
    """u0 = mean + amp sin(2 pi x) sin(2 pi y) + seeded Gaussian noise."""
    X, Y = grid_2d(nx, ny)
    rng = np.random.default_rng(seed)
    u = mean + amp * np.sin(2 * np.pi * X) * np.sin(2 * np.pi * Y)
    if noise:
        u = u + noise * rng.standard_normal((ny, nx))
    return u[None, :, :]


def gaussian_2d(nx, ny, width=100.0):
    """u0 = exp(-width |x - (1/2, 1/2)|^2) (Section 3.3)."""
    X, Y = grid_2d(nx, ny)
    return np.exp(-width * ((X - 0.5) ** 2 + (Y - 0.5) ** 2))[None, :, :]


def linear_sine_2d(nx, ny):
    X, Y = grid_2d(nx, ny)
    return (np.sin(2 * np.pi * X) * np.cos(2 * np.pi * Y))[None, :, :]


def sw_fourier_2d(nx, ny, seed=SEED, modes=8, amp=0.05, h_mean=1.0, kmax=4):
    """(h, hu, hv): h = h_mean + amp sum_m c_m cos(2 pi k_m.x + phi_m), sum |c_m| = 1, at rest."""
    rng = np.random.default_rng(seed)
    X, Y = grid_2d(nx, ny)
    h = np.full((ny, nx), h_mean)
    c = rng.uniform(-1.0, 1.0, modes)
    c /= np.abs(c).sum()
    for m in range(modes):
        while True:
            k = rng.integers(-kmax, kmax + 1, 2)
            if k[0] or k[1]:
                break
        ph = rng.uniform(0.0, 2.0 * np.pi)
        h += amp * c[m] * np.cos(2 * np.pi * (k[0] * X + k[1] * Y) + ph)
    z = np.zeros_like(h)
    return np.stack([h, z, z])


def sw_random_2d(nx, ny, seed=SEED, h_amp=0.05, u_amp=0.05):
    """Smooth (h, hu, hv) with nonzero velocities (for parity tests)."""
    rng = np.random.default_rng(seed)
    X, Y = grid_2d(nx, ny)
    h = 1.0 + h_amp * np.cos(2 * np.pi * (X + 2 * Y) + rng.uniform(0, 6.3))
    u = u_amp * np.sin(2 * np.pi * (2 * X - Y) + rng.uniform(0, 6.3))
    v = u_amp * np.cos(2 * np.pi * (X + Y) + rng.uniform(0, 6.3))
    return np.stack([h, h * u, h * v])


def euler_vortex_2d(nx, ny, length=10.0, strength=5.0, gamma=1.4, u_inf=(1.0, 1.0), centre=(5.0, 5.0)):
    """Isentropic vortex on [0, L]^2 (rho, rho u, rho v, E): background rho = p = 1, velocity u_inf;
    it is advected without change of shape by u_inf."""
    X, Y = grid_2d(nx, ny, length, length)
    dx_, dy_ = X - centre[0], Y - centre[1]
    r2 = dx_ * dx_ + dy_ * dy_
    e = np.exp(0.5 * (1.0 - r2))
    u = u_inf[0] - strength / (2 * np.pi) * e * dy_
    v = u_inf[1] + strength / (2 * np.pi) * e * dx_
    T = 1.0 - (gamma - 1.0) * strength ** 2 / (8 * gamma * np.pi ** 2) * e * e
    rho = T ** (1.0 / (gamma - 1.0))
    p = rho ** gamma
    E = p / (gamma - 1.0) + 0.5 * rho * (u * u + v * v)
    return np.stack([rho, rho * u, rho * v, E])


def euler_riemann_2d(nx, ny, seed=SEED, lo=0.5, hi=1.5, vel=0.5, gamma=1.4):
    """Four constant states with a seeded interface point in [0.3, 0.7]^2 (rho, p in [lo, hi],
    velocities in [-vel, vel])."""
    rng = np.random.default_rng(seed)
    X, Y = grid_2d(nx, ny)
    x0, y0 = rng.uniform(0.3, 0.7, 2)
    out = np.zeros((4, ny, nx))
    for qx in (0, 1):
        for qy in (0, 1):
            rho, p = rng.uniform(lo, hi, 2)
            u, v = rng.uniform(-vel, vel, 2)
            mask = ((X >= x0) == bool(qx)) & ((Y >= y0) == bool(qy))
            out[0][mask] = rho
            out[1][mask] = rho * u
            out[2][mask] = rho * v
            out[3][mask] = p / (gamma - 1.0) + 0.5 * rho * (u * u + v * v)
    return out


def batched_sizes(count=64, lo=256, hi=1024, seed=SEED):
    """Uneven (nx, ny) instance sizes drawn uniformly from [lo, hi]."""
    rng = np.random.default_rng(seed)
    return [(int(a), int(b)) for a, b in rng.integers(lo, hi + 1, size=(count, 2))]


def random_distributions(planes, shape, seed=SEED, scale=1.0):
    """Arbitrary distribution planes (transport-only tests)."""
    rng = np.random.default_rng(seed)
    return scale * rng.standard_normal((planes,) + tuple(shape))


def perturb(f, seed=SEED, scale=1e-3):
    """Move distributions off equilibrium by a seeded perturbation."""
    rng = np.random.default_rng(seed)
    return f + scale * rng.standard_normal(f.shape)


# ---- workloads ----------------------------------------------------------------

def steps_for(t_final, dx, V, step_cells=24, kappa=1):
    """Steps whose lattice time n * (step_cells kappa dx / V) does not exceed t_final,
    with the step length evaluated left to right in double precision."""
    dt = step_cells * kappa * dx / V
    return max(1, int(math.floor(t_final / dt)))


WORKLOADS = {
    # 1D scalar Burgers, D1Q2, N = 256, V = 2 max|u| = 1.5, to t = 0.1
    "burgers1d_n256": dict(dim=1, system="burgers", nx=256, V=1.5, t_final=0.1,
                           init="sine_1d", init_kw=dict(mean=0.5, amp=0.25)),
    # 1D shallow water, D1Q2 per variable, g = 9.81, h0 = 1 + 0.1 sin, at rest, to t = 0.05
    "sw1d": dict(dim=1, system="sw", nx=1 << 20, V=4.0, g=9.81, t_final=0.05,
                 init="sw_sine_1d", init_kw=dict(h_mean=1.0, h_amp=0.1)),
    # 1D shallow-water dam break h in {2, 1}, N = 65536 (V = 6 sqrt(g) from Section 5.2 scaled)
    "sw1d_dambreak": dict(dim=1, system="sw", nx=65536, V=6.0 * math.sqrt(9.81), g=9.81,
                          t_final=0.05, init="sw_dam_break_1d",
                          init_kw=dict(h_left=2.0, h_right=1.0)),
    # 2D scalar Burgers, D2Q4, 4096^2, 2000 composite steps
    "burgers2d_4096": dict(dim=2, system="burgers", nx=4096, ny=4096, V=3.0, steps=2000,
                           init="burgers_2d", init_kw=dict(noise=1e-3)),
}


def make_initial(workload, nx=None, ny=None):
    w = WORKLOADS[workload]
    nx = nx or w["nx"]
    fn = globals()[w["init"]]
    if w["dim"] == 1:
        return fn(nx, **w.get("init_kw", {}))
    return fn(nx, ny or w.get("ny", nx), **w.get("init_kw", {}))
