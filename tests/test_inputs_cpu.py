"""The seeded synthetic inputs (host only): deterministic for a seed, on the grid x_j = j dx, and
with the shapes and value ranges the workloads state."""
import math

import numpy as np

from paper_2403_13406_gb300 import inputs


def test_grids_are_cell_points():
    assert np.allclose(inputs.grid_1d(8), np.arange(8) / 8)
    X, Y = inputs.grid_2d(4, 3)
    assert X.shape == (3, 4) and np.allclose(X[0], np.arange(4) / 4) and np.allclose(Y[:, 0], np.arange(3) / 3)


def test_seeded_generators_are_deterministic():
    for gen in (lambda s: inputs.sw_fourier_2d(16, 12, seed=s), lambda s: inputs.burgers_2d(16, 12, seed=s),
                lambda s: inputs.euler_riemann_2d(16, 12, seed=s), lambda s: inputs.sw_random_1d(32, seed=s)):
        assert np.array_equal(gen(5), gen(5))
        assert not np.array_equal(gen(5), gen(6))


def test_fourier_depth_of_the_batched_workload():
    """h = 1 + 0.05 sum_m c_m cos(2 pi k_m.x + phi_m) with sum |c_m| = 1: |h - 1| <= 0.05, at rest,
    and only wavenumbers |k_j| <= 4 (the spectrum vanishes beyond)."""
    u = inputs.sw_fourier_2d(64, 48, seed=1003)
    assert u.shape == (3, 48, 64)
    assert np.abs(u[0] - 1.0).max() <= 0.05 + 1e-12
    assert not np.any(u[1]) and not np.any(u[2])
    spec = np.abs(np.fft.fft2(u[0] - u[0].mean()))
    ky = np.fft.fftfreq(48, 1 / 48)[:, None]
    kx = np.fft.fftfreq(64, 1 / 64)[None, :]
    assert spec[(np.abs(kx) > 4) | (np.abs(ky) > 4)].max() < 1e-9


def test_batched_sizes_range():
    sizes = inputs.batched_sizes(64, 256, 1024)
    assert len(sizes) == 64 and all(256 <= nx <= 1024 and 256 <= ny <= 1024 for nx, ny in sizes)
    assert sizes == inputs.batched_sizes(64, 256, 1024)


def test_euler_riemann_states_are_admissible():
    u = inputs.euler_riemann_2d(40, 30, seed=9)
    rho, mx, my, E = u
    p = 0.4 * (E - 0.5 * (mx ** 2 + my ** 2) / rho)
    assert rho.min() >= 0.5 and rho.max() <= 1.5 and p.min() >= 0.5 - 1e-12 and p.max() <= 1.5 + 1e-12
    assert len(np.unique(rho)) == 4  # four constant states


def test_vortex_background_and_translation():
    """Far from its centre the isentropic vortex is the background state (rho = p = 1, velocity (1, 1));
    moving the centre by (s, s) translates the field."""
    N = 64
    u = inputs.euler_vortex_2d(N, N)
    assert abs(u[0][0, 0] - 1.0) < 1e-6 and abs(u[1][0, 0] - 1.0) < 1e-6
    shift = 10.0 / N * 8  # eight cells
    v = inputs.euler_vortex_2d(N, N, centre=(5 + shift, 5 + shift))
    # cells whose translate stays inside the grid (the field is not periodic: its tail is ~1e-3 at the edge)
    assert np.allclose(u[:, :-8, :-8], v[:, 8:, 8:], atol=1e-12)


def test_steps_for_floor_reading():
    """n = floor(T / dt) with dt = 24 dx / V in double precision (the Table 6 N = 20 row gives 9)."""
    assert inputs.steps_for(10.0, 1.0 / 20, 1.2) == 9
    assert inputs.steps_for(0.05, 1.0 / (1 << 20), 4.0) == math.floor(0.05 / (24.0 / (1 << 20) / 4.0))
