"""Oracle checks for 2D Euler with a fixed relaxation parameter (Section 6.3).  The paper prints
no Euler values (the Lax-Liu states are external), so parity is pinned by invariants only."""
import math

import numpy as np
import pytest

import oracle as O
from paper_2403_13406_gb300 import inputs


def model(n=24, **kw):
    return O.Model(2, "euler", n, n, V=8.0, gamma=1.4, **kw)


def test_euler_equilibrium_constraints():
    """eq. constraintsKinetic for the Euler fluxes of Section 6.3."""
    m = model()
    rng = np.random.default_rng(1)
    vel = [np.array(v, float) for v in ((1, 0), (0, 1), (-1, 0), (0, -1))]
    for _ in range(5):
        rho, p = rng.uniform(0.5, 1.5, 2)
        u, v = rng.uniform(-0.5, 0.5, 2)
        U = np.array([rho, rho * u, rho * v, p / 0.4 + 0.5 * rho * (u * u + v * v)])
        feq = O.equilibrium(m, U)
        np.testing.assert_allclose(feq.sum(axis=0), U, rtol=1e-15, atol=1e-15)
        phx = np.array([rho * u, rho * u * u + p, rho * u * v, u * (U[3] + p)])
        phy = np.array([rho * v, rho * u * v, rho * v * v + p, v * (U[3] + p)])
        for j, ph in ((0, phx), (1, phy)):
            mom = sum(8.0 * c[j] * feq[k] for k, c in enumerate(vel))
            np.testing.assert_allclose(mom, ph, rtol=1e-13, atol=1e-14)


def test_euler_uniform_state_is_stationary():
    m = model(16)
    U = np.array([1.2, 0.3 * 1.2, -0.2 * 1.2, 1.0 / 0.4 + 0.5 * 1.2 * 0.13])
    u0 = np.broadcast_to(U[:, None, None], (4, 16, 16)).copy()
    f = O.init_equilibrium(m, u0)
    f0 = f.copy()
    O.composite_steps(m, f, 2, scheme="III")
    np.testing.assert_allclose(f, f0, rtol=0, atol=1e-14)


@pytest.mark.parametrize("scheme", ["I", "III"])
def test_euler_vortex_conserves_and_converges(scheme):
    """Mass, momentum and energy are conserved; the advected isentropic vortex error shrinks
    under refinement (Scheme III is the scheme of Section 6.3 for Euler)."""
    errs = []
    for N in (32, 64):
        m = model(N)
        u0 = inputs.euler_vortex_2d(N, N)
        f = O.init_equilibrium(m, u0)
        dx, dt = 10.0 / N, 24 * (10.0 / N) / 8.0
        n = int(round(2.0 / dt))
        O.composite_steps(m, f, n, scheme=scheme)
        u = O.moments(m, f)
        np.testing.assert_allclose(u.sum(axis=(1, 2)), u0.sum(axis=(1, 2)), rtol=1e-12)
        ex = inputs.euler_vortex_2d(N, N, centre=(5 + n * dt, 5 + n * dt))
        errs.append(math.sqrt(float(np.mean((u[0] - ex[0]) ** 2))))
    assert errs[1] < errs[0] / 4


def test_euler_vortex_fourth_order():
    """The isentropic vortex is an exact solution (translated by t (1, 1)): at t = 0.9375 the oracle's
    error falls at fourth order between 128^2 and 256^2 cells (measured 4.43; scheme I, omega = 2)."""
    errs = []
    for N in (128, 256):
        m = model(N)
        u0 = inputs.euler_vortex_2d(N, N)
        f = O.init_equilibrium(m, u0)
        dt = 24 * (10.0 / N) / 8.0
        n = N // 32
        O.composite_steps(m, f, n, scheme="I")
        u = O.moments(m, f)
        ex = inputs.euler_vortex_2d(N, N, centre=(5 + n * dt, 5 + n * dt))
        errs.append(math.sqrt((10.0 / N) ** 2 * float(np.sum((u[0] - ex[0]) ** 2))))
    assert math.log2(errs[0] / errs[1]) > 4.0


@pytest.mark.parametrize("system,kw,mode", [("euler", dict(V=8.0, gamma=1.4), "fixed"),
                                            ("sw", dict(V=8.0, g=9.81), "entropic")])
def test_openmp_build_is_the_same_arithmetic(system, kw, mode):
    """The OpenMP build of the oracle (timed on all host cores as the CPU baseline) splits the cells of a
    relaxation sweep and the planes of a transport over threads: the results are bit for bit those of
    the single-threaded build, and so are the statistics."""
    nx, ny = 48, 40
    u0 = inputs.euler_vortex_2d(nx, ny) if system == "euler" else inputs.sw_random_2d(nx, ny, seed=3, h_amp=0.1)
    out = []
    try:
        for omp in (False, True):
            if not O.set_openmp(omp):
                pytest.skip("no OpenMP in this compiler")
            m = O.Model(2, system, nx, ny, omega_mode=mode, **kw)
            f = O.init_equilibrium(m, u0)
            st = O.Stats()
            O.composite_steps(m, f, 1, stats=st)
            out.append((f, st.as_dict()))
    finally:
        O.set_openmp(False)
    assert np.array_equal(out[0][0], out[1][0])
    assert out[0][1] == out[1][1]
