"""Pins of the oracle's operators and composition (Sections 2.1-2.4, Appendix A)."""
from fractions import Fraction

import numpy as np
import pytest

import oracle as O
from _golden import eval_trace
from paper_2403_13406_gb300 import inputs


def amplification(aV, N, j, scheme="I", V=1.0, omega=2.0):
    """2x2 Fourier symbol of one step of the linear D1Q2 scheme at xi dx = 2 pi j / N, from
    oracle runs on cos and sin initial data (the scheme is linear and translation invariant)."""
    m = O.Model(1, "linear", N, V=V, a=(aV * V, 0.0), omega=omega)
    x = np.arange(N)
    xi = 2 * np.pi * j / N
    A = np.zeros((2, 2), complex)
    for col in range(2):
        for part, fn in ((1.0, np.cos), (1j, np.sin)):
            f = np.zeros((2, N))
            f[col] = fn(xi * x)
            O.composite_steps(m, f, 1, scheme=scheme)
            A[:, col] += part * f[:, 0]
    return A


def test_order_conditions_rational_solution():
    """eqs. fourtOrderConditionOne/Two with n = 4 are solved by alpha = 1/6, beta = -1/3."""
    n, a, b = 4, Fraction(1, 6), Fraction(-1, 3)
    assert 2 * n * a + b == 1
    assert 2 * n * a ** 3 + b ** 3 == 0
    # every transport of psi(alpha dt), psi(beta dt) is an integer number of cells (dt = 24 dx/V)
    for c in (a, b):
        assert (24 * c / 4).denominator == 1 and (24 * c / 2).denominator == 1


@pytest.mark.parametrize("aV", [0.1, 0.3, 0.55, 0.8, 0.95, 0.999])
@pytest.mark.parametrize("N,j", [(8, 1), (12, 1), (16, 3), (10, 3), (20, 7), (64, 5)])
def test_trace_matches_appendix_polynomial(aV, N, j):
    """Appendix A: tr(Phi_hat) is the printed degree-36 polynomial in mu = sin(xi dx), C = 24 a/V."""
    A = amplification(aV, N, j)
    ref = eval_trace(Fraction(24 * aV).limit_denominator(10 ** 12), np.sin(2 * np.pi * j / N))
    assert abs(np.trace(A) - ref) < 1e-11 * max(1.0, abs(ref))
    assert abs(np.linalg.det(A) - 1.0) < 1e-12  # Section 2.4: det = 1 (even number of R)


def test_matrix_at_critical_frequency():
    """Section 2.4: at |a|/V = 1 and xi dx = pi/4 the symbol is [[1, 32 i], [0, 1]]."""
    A = amplification(1.0, 8, 1)
    np.testing.assert_allclose(A, np.array([[1, 32j], [0, 1]]), atol=1e-12)


def test_stability_boundary():
    """Proposition 1: |tr| < 2 below |a| = V; the trace leaves [-2, 2] at mu = sqrt(2)/2 above it."""
    for aV in (0.5, 0.9, 0.99):
        for N, j in ((8, 1), (16, 3), (24, 5)):
            assert abs(np.trace(amplification(aV, N, j)).real) <= 2.0 + 1e-12
    assert abs(np.trace(amplification(1.05, 8, 1)).real) > 2.0


def test_exact_shift_when_a_equals_V():
    """a = V: f^eq_- = 0 and every R_2 maps (u, 0) to itself, so one composite step is the exact
    shift by V dt / dx = 24 cells (Section 2.3, dt = 24 kappa dx / V), bit for bit."""
    N = 97
    m = O.Model(1, "linear", N, V=2.0, a=(2.0, 0.0))  # a u / (2V) = u/2 exactly
    u0 = inputs.random_scalar_1d(N, seed=3)
    f = O.init_equilibrium(m, u0)
    done = 0
    for n in (1, 2, 5):
        O.composite_steps(m, f, n)
        done += n
        u = O.moments(m, f)[0]
        assert np.array_equal(u, np.roll(u0[0], 24 * done))


@pytest.mark.parametrize("system,kw", [("burgers", dict(V=1.5)), ("sw", dict(V=6.0, g=9.81)),
                                       ("linear", dict(V=1.0, a=(0.3, 0.0)))])
@pytest.mark.parametrize("mode", ["fixed", "entropic"])
def test_brick_is_time_symmetric_1d(system, kw, mode):
    """eq. symmetryCondition: psi(dt) psi(-dt) = Id for the brick of eq. basicBrickSplitting (both
    with omega = 2 and with the entropic omega, whose relaxation is an involution, Section 4)."""
    N = 40
    m = O.Model(1, system, N, omega_mode=mode, **kw)
    u0 = inputs.sw_random_1d(N, seed=5) if system == "sw" else inputs.random_scalar_1d(N, seed=5)
    f0 = inputs.perturb(O.init_equilibrium(m, u0), seed=9, scale=1e-3)
    f = f0.copy()
    O.brick(m, f, 1, 6)   # psi(dt/6): shifts 1, 2, 1
    O.brick(m, f, -1, 6)  # psi(-dt/6)
    tol = 1e-13 if mode == "fixed" else 1e-11
    np.testing.assert_allclose(f, f0, rtol=0, atol=tol)


@pytest.mark.parametrize("system,kw", [("burgers", dict(V=3.0, c=(1.0, 0.6))), ("sw", dict(V=10.0, g=9.81))])
def test_brick_is_time_symmetric_2d(system, kw):
    m = O.Model(2, system, 12, 10, omega_mode="entropic", **kw)
    u0 = inputs.sw_random_2d(12, 10, seed=2) if system == "sw" else inputs.burgers_2d(12, 10, seed=2, noise=0)
    f0 = inputs.perturb(O.init_equilibrium(m, u0), seed=4, scale=1e-4)
    f = f0.copy()
    O.brick(m, f, -1, 3)
    O.brick(m, f, 1, 3)
    np.testing.assert_allclose(f, f0, rtol=0, atol=1e-11)


@pytest.mark.parametrize("dim", [1, 2])
def test_transport_is_a_permutation(dim):
    """eq. transportPhase: shifts only; T(s) T(-s) = Id bit for bit, values of every plane are
    permuted, and the total microscopic entropy is unchanged (Section 4)."""
    if dim == 1:
        m = O.Model(1, "sw", 33, V=6.0, g=9.81)
        u0 = inputs.sw_random_1d(33, seed=1)
    else:
        m = O.Model(2, "sw", 9, 7, V=10.0, g=9.81)
        u0 = inputs.sw_random_2d(9, 7, seed=1)
    f0 = inputs.perturb(O.init_equilibrium(m, u0), seed=1, scale=1e-3)
    for s in (1, 2, -4, 5):
        f = f0.copy()
        O.transport(m, f, s)
        for pl in range(f.shape[0]):
            assert np.array_equal(np.sort(f[pl].ravel()), np.sort(f0[pl].ravel()))
        assert np.isclose(O.entropy_totals(m, f)[0], O.entropy_totals(m, f0)[0], rtol=1e-13)
        O.transport(m, f, -s)
        assert np.array_equal(f, f0)


def test_transport_direction():
    """f_k(x) <- f_k(x - kappa V_k/V dx): the + population moves right, the - population left."""
    m = O.Model(1, "burgers", 8, V=1.0)
    f = np.zeros((2, 8))
    f[0, 2] = 1.0
    f[1, 2] = 2.0
    O.transport(m, f, 3)
    assert f[0, 5] == 1.0 and f[1, 7] == 2.0
    m2 = O.Model(2, "burgers", 6, 5, V=1.0)
    g = np.zeros((4, 5, 6))
    for k in range(4):
        g[k, 2, 2] = k + 1
    O.transport(m2, g, 1)
    assert g[0, 2, 3] == 1 and g[1, 3, 2] == 2 and g[2, 2, 1] == 3 and g[3, 1, 2] == 4


def test_step_lengths():
    """dt = 24 kappa dx / V for the composite schemes; scheme (B) of Section 6.3 uses 4 dx / V and
    the standard scheme R T one cell."""
    m = O.Model(1, "burgers", 8, V=1.0)
    assert O.step_length(m, "I") == 24 and O.step_length(m, "plain") == 1
    assert O.step_length(m, "B") == 4


@pytest.mark.parametrize("aV", [0.2, 0.45, 0.7])
def test_scheme_b_symbol_is_second_order(aV):
    """Section 6.3, scheme (B) = R_1 T(dt/4) R_2 T(dt/2) R_2 T(dt/4) with dt = 4 dx / V.  On linear
    D1Q2 its symbol has rank one (R_1 is the last operator) and the non-zero eigenvalue, worked out
    from the operator definitions (T(s) multiplies f_+ by exp(-i s xi dx) and f_- by exp(i s xi dx),
    R_2 f = 2 f^eq(u) - f, R_1 f = f^eq(u)), is
        z = exp(-i a xi dt) + a (V^2 - a^2) / 24 * (i (xi dt)^3 + a (xi dt)^4) + O((xi dt)^5)
    (V = 1 here): a second-order scheme whose leading error vanishes at a = 0 and |a| = V.  A wrong
    shift (1, 2, 1 cells) or a relaxation left out changes the cubic coefficient."""
    V, N = 1.0, 400
    for j in (1, 2):
        A = amplification(aV, N, j, scheme="B", V=V)
        ev = np.linalg.eigvals(A)
        assert min(np.abs(ev)) < 1e-12
        z = ev[np.argmax(np.abs(ev))]
        xdt = 2 * np.pi * j / N * 4 / V
        k3 = 1j * aV * (V ** 2 - aV ** 2) / 24
        k4 = aV ** 2 * (V ** 2 - aV ** 2) / 24
        d = z - np.exp(-1j * aV * xdt)
        assert abs(d.imag / xdt ** 3 - k3.imag) < 2e-2 * abs(k3)
        assert abs(d.real / xdt ** 4 - k4) < 5e-2 * abs(k4)


@pytest.mark.parametrize("system,kw", [("burgers", dict(V=2.0)), ("sw", dict(V=4.0, g=1.0))])
def test_scheme_b_ends_with_the_projection(system, kw):
    """Scheme (B) applies R_1 last (Section 6.3: one basic brick plus a relaxation on the equilibrium),
    so the distributions after every step are at equilibrium, f = f^eq(u), whatever the initial data.
    A symbol test cannot see where R_1 sits (R_1 A and A R_1 share their non-zero eigenvalue); this
    one fails if R_1 is moved."""
    N = 64
    m = O.Model(1, system, N, **kw)
    u0 = inputs.sw_random_1d(N, seed=4) if system == "sw" else inputs.random_scalar_1d(N, seed=4)
    f = inputs.perturb(O.init_equilibrium(m, u0), seed=5, scale=0.02)
    f_eq0 = O.init_equilibrium(m, O.moments(m, f))
    assert np.abs(f - f_eq0).max() > 1e-4  # the start is off equilibrium
    for _ in range(3):
        O.composite_steps(m, f, 1, scheme="B")
        f_eq = O.init_equilibrium(m, O.moments(m, f))
        np.testing.assert_allclose(f, f_eq, rtol=0, atol=1e-14)
