"""FP64 CPU oracle of the fourth-order entropy-stable lattice Boltzmann scheme.

TEST INFRASTRUCTURE ONLY: the slow, literal restatement of the method
(Bellotti, Helluy, Navoret, arXiv 2403.13406) that the CUDA path is checked
against.  Only tests/, ``__graft_entry__.smoke()`` and the cpu_baseline /
reference legs of ``bench.py`` may import it.  It shares no code with the
CUDA library and never imports the product package.

Arrays: distributions ``f`` have shape ``(q*M, ny, nx)`` (``(q*M, nx)`` in 1D),
plane ``k*M + m``; conserved fields ``u`` have shape ``(M, ny, nx)``.
"""
import ctypes
import numpy as np

from . import build as _build

LINEAR, BURGERS, SW, EULER = 0, 1, 2, 3
SYSTEMS = {"linear": LINEAR, "burgers": BURGERS, "sw": SW, "shallow_water": SW, "euler": EULER}
FIXED, ENTROPIC = 0, 1
R_MAIN, R_PROJECT = 0, 1
SCHEMES = {"I": 1, "II": 2, "III": 3, "IV": 4, "plain": 5, "B": 6}


class _Model(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int), ("system", ctypes.c_int),
                ("nx", ctypes.c_long), ("ny", ctypes.c_long),
                ("kappa", ctypes.c_int), ("V", ctypes.c_double),
                ("a", ctypes.c_double * 2), ("c", ctypes.c_double * 2),
                ("g", ctypes.c_double), ("omega_mode", ctypes.c_int),
                ("omega", ctypes.c_double), ("t_max", ctypes.c_double), ("gamma", ctypes.c_double)]


class Stats(ctypes.Structure):
    _fields_ = [("relaxations", ctypes.c_long), ("fallbacks", ctypes.c_long),
                ("omega_min", ctypes.c_double), ("omega_max", ctypes.c_double)]

    def __init__(self):
        super().__init__(0, 0, float("inf"), float("-inf"))

    def as_dict(self):
        return {"relaxations": self.relaxations, "fallbacks": self.fallbacks,
                "omega_min": self.omega_min, "omega_max": self.omega_max}


_libs = {}
_openmp = False
_D = ctypes.POINTER(ctypes.c_double)


def set_openmp(enable):
    """Route later calls to the OpenMP build (cells and planes split over the host cores, the same
    per-cell arithmetic) or back to the single-threaded one.  Returns False, and stays
    single-threaded, where the compiler has no OpenMP."""
    global _openmp
    if enable and _build.build_openmp() is None:
        _openmp = False
        return False
    _openmp = bool(enable)
    return True


def lib():
    key = "omp" if _openmp else "single"
    if key not in _libs:
        L = ctypes.CDLL(_build.build_openmp() if _openmp else _build.build())
        P = ctypes.POINTER(_Model)
        S = ctypes.POINTER(Stats)
        sig = {
            "or_q": (ctypes.c_int, [P]), "or_M": (ctypes.c_int, [P]),
            "or_ncell": (ctypes.c_long, [P]), "or_check": (ctypes.c_int, [P]),
            "or_flux": (None, [P, ctypes.c_int, _D, _D]),
            "or_entropy_S": (ctypes.c_double, [P, _D]),
            "or_dual": (None, [P, _D, _D]),
            "or_equilibrium": (None, [P, _D, _D]),
            "or_kinetic_dual": (ctypes.c_double, [P, ctypes.c_int, _D, _D, _D]),
            "or_kinetic_entropy": (ctypes.c_double, [P, ctypes.c_int, _D, _D]),
            "or_bregman": (ctypes.c_double, [P, ctypes.c_int, _D, _D, _D]),
            "or_entropy_imbalance": (ctypes.c_double, [P, _D, ctypes.c_double]),
            "or_omega": (ctypes.c_double, [P, _D, S]),
            "or_init_equilibrium": (None, [P, _D, _D]),
            "or_transport": (ctypes.c_int, [P, _D, ctypes.c_long]),
            "or_relax": (ctypes.c_int, [P, _D, ctypes.c_int, S]),
            "or_brick": (ctypes.c_int, [P, _D, ctypes.c_long, ctypes.c_long, S]),
            "or_composite_steps": (ctypes.c_int, [P, _D, ctypes.c_int, ctypes.c_long, S]),
            "or_step_length": (ctypes.c_long, [P, ctypes.c_int]),
            "or_moments": (None, [P, _D, _D]),
            "or_entropy_totals": (None, [P, _D, _D, _D]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _libs[key] = L
    return _libs[key]


def _ptr(a):
    return a.ctypes.data_as(_D)


def _vec(x, n):
    a = np.zeros(n, dtype=np.float64)
    a[: len(x)] = x
    return a


class Model:
    """Parameters of one run: velocity set, system, grid and relaxation.

    ``dim`` 1 selects D1Q2, 2 selects D2Q4 (Section 1.2).  ``omega`` is the
    relaxation parameter in fixed mode; ``omega_mode='entropic'`` selects the
    per-cell root of eq. variableOmegaProblem.
    """

    def __init__(self, dim, system, nx, ny=1, V=1.0, a=(0.0, 0.0), c=(1.0, 1.0), g=1.0,
                 omega_mode="fixed", omega=2.0, t_max=3.0, kappa=1, gamma=1.4):
        self.dim = int(dim)
        self.system = SYSTEMS[system] if isinstance(system, str) else int(system)
        self.nx, self.ny = int(nx), (int(ny) if dim == 2 else 1)
        self.V = float(V)
        self.c_struct = _Model(self.dim, self.system, self.nx, self.ny, int(kappa), self.V,
                               (ctypes.c_double * 2)(*a), (ctypes.c_double * 2)(*c), float(g),
                               ENTROPIC if omega_mode == "entropic" else FIXED,
                               float(omega), float(t_max), float(gamma))
        if lib().or_check(ctypes.byref(self.c_struct)) != 0:
            raise ValueError("invalid oracle model")
        self.q = lib().or_q(ctypes.byref(self.c_struct))
        self.M = lib().or_M(ctypes.byref(self.c_struct))

    @property
    def ref(self):
        return ctypes.byref(self.c_struct)

    @property
    def grid_shape(self):
        return (self.nx,) if self.dim == 1 else (self.ny, self.nx)

    @property
    def ncell(self):
        return self.nx * self.ny

    def with_(self, **kw):
        s = self.c_struct
        base = dict(dim=self.dim, system=self.system, nx=self.nx, ny=self.ny, V=s.V,
                    a=tuple(s.a), c=tuple(s.c), g=s.g,
                    omega_mode="entropic" if s.omega_mode == ENTROPIC else "fixed",
                    omega=s.omega, t_max=s.t_max, kappa=s.kappa, gamma=s.gamma)
        base.update(kw)
        return Model(**base)


def _fshape(m):
    return (m.q * m.M,) + m.grid_shape


def _check_f(m, f):
    if f.dtype != np.float64 or not f.flags.c_contiguous or f.shape != _fshape(m):
        raise ValueError("f must be a C-contiguous float64 array of shape %s" % (_fshape(m),))


# ---- per-cell quantities ---------------------------------------------------

def flux(m, j, u):
    u = _vec(u, 4)
    out = np.zeros(4)
    lib().or_flux(m.ref, j, _ptr(u), _ptr(out))
    return out[: m.M]


def dual(m, u):
    u = _vec(u, 4)
    p = np.zeros(4)
    lib().or_dual(m.ref, _ptr(u), _ptr(p))
    return p[: m.M]


def entropy_S(m, u):
    return lib().or_entropy_S(m.ref, _ptr(_vec(u, 4)))


def equilibrium(m, u):
    """f^eq_k(u) for one cell, shape (q, M)."""
    out = np.zeros(16)
    lib().or_equilibrium(m.ref, _ptr(_vec(u, 4)), _ptr(out))
    return out[: m.q * m.M].reshape(m.q, m.M)


def kinetic_dual(m, k, p):
    """(s*_k(p), grad, Hessian)."""
    gr = np.zeros(3)
    H = np.zeros(9)
    v = lib().or_kinetic_dual(m.ref, k, _ptr(_vec(p, 3)), _ptr(gr), _ptr(H))
    M = m.M
    return v, gr[:M].copy(), H[: M * M].reshape(M, M).copy()


def kinetic_entropy(m, k, fk, p_hint):
    return lib().or_kinetic_entropy(m.ref, k, _ptr(_vec(fk, 3)), _ptr(_vec(p_hint, 3)))


def bregman(m, k, u, h):
    """(B_k(h), Delta) around the equilibrium of u."""
    D = np.zeros(3)
    b = lib().or_bregman(m.ref, k, _ptr(_vec(u, 3)), _ptr(_vec(h, 3)), _ptr(D))
    return b, D[: m.M].copy()


def _cell(m, fcell):
    fc = np.ascontiguousarray(np.asarray(fcell, dtype=np.float64).reshape(-1))
    if fc.size != m.q * m.M:
        raise ValueError("cell state must have q*M entries")
    return fc


def entropy_imbalance(m, fcell, omega):
    return lib().or_entropy_imbalance(m.ref, _ptr(_cell(m, fcell)), float(omega))


def omega(m, fcell, stats=None):
    st = stats if stats is not None else Stats()
    return lib().or_omega(m.ref, _ptr(_cell(m, fcell)), ctypes.byref(st))


# ---- grid operators ----------------------------------------------------------

def init_equilibrium(m, u0):
    u0 = np.ascontiguousarray(u0, dtype=np.float64).reshape((m.M,) + m.grid_shape)
    f = np.zeros(_fshape(m))
    lib().or_init_equilibrium(m.ref, _ptr(u0), _ptr(f))
    return f


def transport(m, f, s):
    _check_f(m, f)
    if lib().or_transport(m.ref, _ptr(f), int(s)):
        raise RuntimeError("transport failed")
    return f


def relax(m, f, kind=R_MAIN, stats=None):
    _check_f(m, f)
    st = stats if stats is not None else Stats()
    lib().or_relax(m.ref, _ptr(f), int(kind), ctypes.byref(st))
    return f


def brick(m, f, num, den, stats=None):
    _check_f(m, f)
    st = stats if stats is not None else Stats()
    if lib().or_brick(m.ref, _ptr(f), int(num), int(den), ctypes.byref(st)):
        raise ValueError("brick shifts are not integers")
    return f


def composite_steps(m, f, nsteps=1, scheme="I", stats=None):
    _check_f(m, f)
    st = stats if stats is not None else Stats()
    if lib().or_composite_steps(m.ref, _ptr(f), SCHEMES[scheme], int(nsteps), ctypes.byref(st)):
        raise RuntimeError("composite step failed")
    return f


def step_length(m, scheme="I"):
    """Lattice units (dx/V) advanced by one step of the scheme."""
    return lib().or_step_length(m.ref, SCHEMES[scheme])


def time_step(m, dx, scheme="I"):
    """dt of one step: 24 kappa dx / V for the composite schemes (Section 2.3)."""
    return step_length(m, scheme) * dx / m.V


def moments(m, f):
    _check_f(m, f)
    u = np.zeros((m.M,) + m.grid_shape)
    lib().or_moments(m.ref, _ptr(f), _ptr(u))
    return u


def entropy_totals(m, f):
    _check_f(m, f)
    s = ctypes.c_double()
    S = ctypes.c_double()
    lib().or_entropy_totals(m.ref, _ptr(f), ctypes.byref(s), ctypes.byref(S))
    return s.value, S.value
