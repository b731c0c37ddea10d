"""Thin ctypes binding of the C ABI in include/eslbm.h.

Argument marshalling only: every step of the composite scheme runs in the
sm_103a kernels of libeslbm.so.  PyTorch provides device memory (the two state
buffers and the workspace are torch tensors) and the CUDA stream.  There is no
CPU fallback: if the library has not been built, loading it raises.
"""
import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libeslbm.so")

OK, ERR_ARG, ERR_DOMAIN, ERR_CUDA, ERR_NAN, ERR_UNSUPPORTED, WARN_OMEGA_FALLBACK = 0, 1, 2, 3, 4, 5, 100
LINEAR, BURGERS, SHALLOW_WATER, EULER = 0, 1, 2, 3
SYSTEMS = {"linear": LINEAR, "burgers": BURGERS, "sw": SHALLOW_WATER, "shallow_water": SHALLOW_WATER,
           "euler": EULER}
FP32, FP64, FP32_MIXED = 0, 1, 2
PRECISIONS = {"fp32": FP32, "fp64": FP64, "float64": FP64, "fp32_mixed": FP32_MIXED}
BLOCKING_AUTO, BLOCKING_OFF = 0, 1
OMEGA_FIXED, OMEGA_ENTROPIC = 0, 1
SCHEMES = {"I": 1, "II": 2, "III": 3, "IV": 4, "plain": 5, "B": 6}
RELAX_MAIN, RELAX_PROJECT = 0, 1

EXPORTS = ("eslbm_abi_version", "eslbm_status_string", "eslbm_query", "eslbm_create", "eslbm_destroy",
           "eslbm_set_stream", "eslbm_last_error", "eslbm_init_equilibrium", "eslbm_init_distributions",
           "eslbm_step", "eslbm_transport", "eslbm_relax", "eslbm_read_moments", "eslbm_read_distributions",
           "eslbm_read_totals", "eslbm_get_diagnostics", "eslbm_reset_diagnostics", "eslbm_use_graph",
           "eslbm_read_totals_noalloc", "eslbm_gradient_workspace", "eslbm_gradient",
           "eslbm_batch_query", "eslbm_batch_create", "eslbm_batch_destroy", "eslbm_batch_last_error",
           "eslbm_batch_init_equilibrium", "eslbm_batch_step", "eslbm_batch_read_moments",
           "eslbm_batch_set_schedule", "eslbm_batch_get_schedule", "eslbm_batch_tune", "eslbm_batch_use_graph",
           "eslbm_batch_gradient_workspace", "eslbm_batch_gradient", "eslbm_batch_get_diagnostics")


class Config(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int32), ("system", ctypes.c_int32), ("precision", ctypes.c_int32),
                ("omega_mode", ctypes.c_int32), ("scheme", ctypes.c_int32), ("kappa", ctypes.c_int32),
                ("nx", ctypes.c_int64), ("ny", ctypes.c_int64), ("V", ctypes.c_double),
                ("omega", ctypes.c_double), ("a", ctypes.c_double * 2), ("c", ctypes.c_double * 2),
                ("g", ctypes.c_double), ("gamma", ctypes.c_double), ("t_max", ctypes.c_double),
                ("diagnostics", ctypes.c_int32), ("shifted", ctypes.c_int32), ("u_ref", ctypes.c_double * 4),
                ("blocking", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class Sizes(ctypes.Structure):
    _fields_ = [("q", ctypes.c_int64), ("M", ctypes.c_int64), ("planes", ctypes.c_int64),
                ("ncell", ctypes.c_int64), ("state_bytes", ctypes.c_uint64),
                ("workspace_bytes", ctypes.c_uint64), ("stages_per_step", ctypes.c_int64),
                ("step_cells", ctypes.c_int64), ("launches_per_step", ctypes.c_double)]


class Diagnostics(ctypes.Structure):
    _fields_ = [("relaxations", ctypes.c_uint64), ("fallbacks", ctypes.c_uint64),
                ("entropy_increases", ctypes.c_uint64), ("omega_min", ctypes.c_double),
                ("omega_max", ctypes.c_double), ("entropy_excess_max", ctypes.c_double)]


class BatchSizes(ctypes.Structure):
    _fields_ = [("count", ctypes.c_int32), ("q", ctypes.c_int64), ("M", ctypes.c_int64),
                ("planes", ctypes.c_int64), ("total_cells", ctypes.c_int64), ("pool_bytes", ctypes.c_uint64),
                ("workspace_bytes", ctypes.c_uint64), ("stages_per_step", ctypes.c_int64),
                ("step_cells", ctypes.c_int64)]


_lib = None


def lib():
    """Load libeslbm.so (built by __graft_entry__.build() or build.py); raises if absent."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError("libeslbm.so is not built (%s); run paper_2403_13406_gb300/build.py" % LIB_PATH)
    L = ctypes.CDLL(LIB_PATH)
    vp, i32, i64, D = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.POINTER(ctypes.c_double)
    H = ctypes.c_void_p
    sig = {
        "eslbm_abi_version": (i32, []),
        "eslbm_status_string": (ctypes.c_char_p, [ctypes.c_int]),
        "eslbm_query": (ctypes.c_int, [ctypes.POINTER(Config), ctypes.POINTER(Sizes)]),
        "eslbm_create": (ctypes.c_int, [ctypes.POINTER(Config), vp, vp, vp, vp, ctypes.POINTER(H)]),
        "eslbm_destroy": (ctypes.c_int, [H]),
        "eslbm_set_stream": (ctypes.c_int, [H, vp]),
        "eslbm_last_error": (ctypes.c_char_p, [H]),
        "eslbm_init_equilibrium": (ctypes.c_int, [H, vp, i32]),
        "eslbm_init_distributions": (ctypes.c_int, [H, vp, i32]),
        "eslbm_step": (ctypes.c_int, [H, i64]),
        "eslbm_transport": (ctypes.c_int, [H, i64]),
        "eslbm_relax": (ctypes.c_int, [H, i32]),
        "eslbm_read_moments": (ctypes.c_int, [H, vp, i32]),
        "eslbm_read_distributions": (ctypes.c_int, [H, vp, i32]),
        "eslbm_read_totals": (ctypes.c_int, [H, vp, i32]),
        "eslbm_get_diagnostics": (ctypes.c_int, [H, ctypes.POINTER(Diagnostics)]),
        "eslbm_reset_diagnostics": (ctypes.c_int, [H]),
        "eslbm_use_graph": (ctypes.c_int, [H, i32]),
        "eslbm_read_totals_noalloc": (ctypes.c_int, [ctypes.POINTER(Config), vp, i64, vp, i32, vp]),
        "eslbm_gradient_workspace": (ctypes.c_int, [ctypes.POINTER(Config), i64, i64,
                                                    ctypes.POINTER(ctypes.c_uint64)]),
        "eslbm_gradient": (ctypes.c_int, [H, vp, vp, vp, i64, i64, vp, ctypes.c_uint64]),
        "eslbm_batch_query": (ctypes.c_int, [ctypes.POINTER(Config), i32, vp, vp, ctypes.POINTER(BatchSizes)]),
        "eslbm_batch_create": (ctypes.c_int, [ctypes.POINTER(Config), i32, vp, vp, vp, vp, vp, vp,
                                              ctypes.POINTER(H)]),
        "eslbm_batch_destroy": (ctypes.c_int, [H]),
        "eslbm_batch_last_error": (ctypes.c_char_p, [H]),
        "eslbm_batch_init_equilibrium": (ctypes.c_int, [H, vp, i32]),
        "eslbm_batch_step": (ctypes.c_int, [H, i64]),
        "eslbm_batch_read_moments": (ctypes.c_int, [H, vp, i32]),
        "eslbm_batch_set_schedule": (ctypes.c_int, [H, i64, i32, i32]),
        "eslbm_batch_get_schedule": (ctypes.c_int, [H, ctypes.POINTER(i64), ctypes.POINTER(i32),
                                                    ctypes.POINTER(i32)]),
        "eslbm_batch_tune": (ctypes.c_int, [H, vp, ctypes.c_uint64, i32]),
        "eslbm_batch_use_graph": (ctypes.c_int, [H, i32]),
        "eslbm_batch_gradient_workspace": (ctypes.c_int, [ctypes.POINTER(Config), i32, vp, vp, i64, i64,
                                                          ctypes.POINTER(ctypes.c_uint64)]),
        "eslbm_batch_gradient": (ctypes.c_int, [H, vp, vp, vp, i64, i64, vp, ctypes.c_uint64]),
        "eslbm_batch_get_diagnostics": (ctypes.c_int, [H, ctypes.POINTER(Diagnostics)]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    _lib = L
    return L


class EslbmError(RuntimeError):
    def __init__(self, status, message):
        super().__init__(message)
        self.status = status


def make_config(dim, system, nx, ny=1, V=1.0, precision="fp32", omega_mode="fixed", omega=2.0, scheme="I",
                a=(0.0, 0.0), c=(1.0, 1.0), g=1.0, gamma=1.4, t_max=3.0, kappa=1, diagnostics=False, u_ref=None,
                blocking=True):
    """Configuration of one lattice; u_ref (conserved values) selects the shifted storage; precision is
    "fp32", "fp64" or "fp32_mixed"; blocking=False runs one launch per fused stage, an int n >= 2 at
    most n stages per temporally blocked 2D launch."""
    cfg = Config()
    cfg.dim = int(dim)
    cfg.system = SYSTEMS[system] if isinstance(system, str) else int(system)
    cfg.precision = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
    cfg.omega_mode = OMEGA_ENTROPIC if omega_mode in ("entropic", OMEGA_ENTROPIC) else OMEGA_FIXED
    cfg.scheme = SCHEMES[scheme] if isinstance(scheme, str) else int(scheme)
    cfg.kappa = int(kappa)
    cfg.nx = int(nx)
    cfg.ny = int(ny) if dim == 2 else 1
    cfg.V = float(V)
    cfg.omega = float(omega)
    cfg.a[0], cfg.a[1] = float(a[0]), float(a[1])
    cfg.c[0], cfg.c[1] = float(c[0]), float(c[1])
    cfg.g = float(g)
    cfg.gamma = float(gamma)
    cfg.t_max = float(t_max)
    cfg.diagnostics = 1 if diagnostics else 0
    cfg.shifted = 0 if u_ref is None else 1
    if blocking is True or blocking is None:
        cfg.blocking = BLOCKING_AUTO
    elif blocking is False:
        cfg.blocking = BLOCKING_OFF
    else:
        cfg.blocking = int(blocking)  # at most this many stages per 2D launch
    if u_ref is not None:
        for i, v in enumerate(u_ref):
            cfg.u_ref[i] = float(v)
    return cfg


def query(cfg):
    sz = Sizes()
    st = lib().eslbm_query(ctypes.byref(cfg), ctypes.byref(sz))
    if st != OK:
        raise EslbmError(st, lib().eslbm_status_string(st).decode())
    return sz


def read_totals_noalloc(cfg, f_ptr, pending_shift, out, out_on_device, stream_handle):
    """Totals of a caller-held state without any allocation (see include/eslbm.h)."""
    st = lib().eslbm_read_totals_noalloc(ctypes.byref(cfg), f_ptr, int(pending_shift), out, int(out_on_device),
                                         stream_handle)
    if st != OK:
        raise EslbmError(st, lib().eslbm_status_string(st).decode())


class Simulation:
    """One lattice, its two state buffers and workspace (torch CUDA tensors), and a handle."""

    def __init__(self, cfg, stream=None, device=None):
        import torch
        self.torch = torch
        self.cfg = cfg
        self.sizes = query(cfg)
        self.device = torch.device(device or "cuda")
        nb = int(self.sizes.state_bytes)
        self._fa = torch.empty(nb, dtype=torch.uint8, device=self.device)
        self._fb = torch.empty(nb, dtype=torch.uint8, device=self.device)
        self._ws = torch.empty(int(self.sizes.workspace_bytes), dtype=torch.uint8, device=self.device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        h = ctypes.c_void_p()
        self._check(lib().eslbm_create(ctypes.byref(cfg), self._fa.data_ptr(), self._fb.data_ptr(),
                                       self._ws.data_ptr(), self.stream.cuda_stream, ctypes.byref(h)), None)
        self.h = h

    # -- shapes ------------------------------------------------------------
    @property
    def grid_shape(self):
        return (self.cfg.nx,) if self.cfg.dim == 1 else (self.cfg.ny, self.cfg.nx)

    @property
    def M(self):
        return int(self.sizes.M)

    @property
    def planes(self):
        return int(self.sizes.planes)

    def _check(self, st, h=True):
        if st in (OK, WARN_OMEGA_FALLBACK):
            return st
        msg = lib().eslbm_status_string(st).decode()
        if h is not None and getattr(self, "h", None) is not None:
            msg += ": " + lib().eslbm_last_error(self.h).decode()
        raise EslbmError(st, msg)

    def close(self):
        if getattr(self, "h", None) is not None:
            lib().eslbm_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- buffers -------------------------------------------------------------
    def _in(self, arr, shape):
        """(pointer, on_device, keepalive) for a double input given as a CUDA tensor or host array."""
        torch = self.torch
        if isinstance(arr, torch.Tensor) and arr.is_cuda:
            t = arr.to(torch.float64).contiguous().reshape(shape)
            return t.data_ptr(), 1, t
        a = np.ascontiguousarray(np.asarray(arr, dtype=np.float64).reshape(shape))
        return a.ctypes.data, 0, a

    # -- ABI calls -------------------------------------------------------------
    def init_equilibrium(self, u0):
        p, dev, keep = self._in(u0, (self.M,) + self.grid_shape)
        return self._check(lib().eslbm_init_equilibrium(self.h, p, dev))

    def init_distributions(self, f0):
        p, dev, keep = self._in(f0, (self.planes,) + self.grid_shape)
        return self._check(lib().eslbm_init_distributions(self.h, p, dev))

    def step(self, n=1):
        return self._check(lib().eslbm_step(self.h, int(n)))

    def transport(self, s):
        return self._check(lib().eslbm_transport(self.h, int(s)))

    def relax(self, kind=RELAX_MAIN):
        return self._check(lib().eslbm_relax(self.h, int(kind)))

    def use_graph(self, enable=True):
        return self._check(lib().eslbm_use_graph(self.h, 1 if enable else 0))

    def set_stream(self, stream):
        self.stream = stream
        return self._check(lib().eslbm_set_stream(self.h, stream.cuda_stream))

    def moments(self, host=False, out=None):
        shape = (self.M,) + self.grid_shape
        if host:
            a = np.empty(shape, dtype=np.float64)
            self._check(lib().eslbm_read_moments(self.h, a.ctypes.data, 0))
            return a
        t = out if out is not None else self.torch.empty(shape, dtype=self.torch.float64, device=self.device)
        self._check(lib().eslbm_read_moments(self.h, t.data_ptr(), 1))
        return t

    def distributions(self, host=False):
        shape = (self.planes,) + self.grid_shape
        if host:
            a = np.empty(shape, dtype=np.float64)
            self._check(lib().eslbm_read_distributions(self.h, a.ctypes.data, 0))
            return a
        t = self.torch.empty(shape, dtype=self.torch.float64, device=self.device)
        self._check(lib().eslbm_read_distributions(self.h, t.data_ptr(), 1))
        return t

    def totals(self, host=True, out=None):
        """[sum Sigma(f), sum S(u), sum u_1, ..., sum u_M] in double precision."""
        n = 2 + self.M
        if host:
            a = np.empty(n, dtype=np.float64)
            self._check(lib().eslbm_read_totals(self.h, a.ctypes.data, 0))
            return a
        t = out if out is not None else self.torch.empty(n, dtype=self.torch.float64, device=self.device)
        self._check(lib().eslbm_read_totals(self.h, t.data_ptr(), 1))
        return t

    def diagnostics(self):
        d = Diagnostics()
        st = lib().eslbm_get_diagnostics(self.h, ctypes.byref(d))
        self._check(st)
        return {"relaxations": d.relaxations, "fallbacks": d.fallbacks,
                "entropy_increases": d.entropy_increases, "omega_min": d.omega_min, "omega_max": d.omega_max,
                "entropy_excess_max": d.entropy_excess_max, "status": st}

    def reset_diagnostics(self):
        return self._check(lib().eslbm_reset_diagnostics(self.h))

    def gradient(self, u0, dJ_duT, n, K=50):
        """dJ/du0 (CUDA float64 tensor) for the moments after n steps from equilibrium at u0,
        given the cotangent dJ/du_T; checkpoints every K steps (the workspace is a torch tensor)."""
        torch = self.torch
        nb = ctypes.c_uint64()
        st = lib().eslbm_gradient_workspace(ctypes.byref(self.cfg), int(n), int(K), ctypes.byref(nb))
        self._check(st)
        ws = torch.empty(int(nb.value) + 256, dtype=torch.uint8, device=self.device)
        ptr = (ws.data_ptr() + 255) // 256 * 256
        shape = (self.M,) + self.grid_shape
        u0 = u0.to(device=self.device, dtype=torch.float64).contiguous().reshape(shape)
        g = dJ_duT.to(device=self.device, dtype=torch.float64).contiguous().reshape(shape)
        out = torch.empty(shape, dtype=torch.float64, device=self.device)
        self._check(lib().eslbm_gradient(self.h, u0.data_ptr(), g.data_ptr(), out.data_ptr(), int(n), int(K), ptr,
                                         nb.value))
        return out


def _aligned(torch, nbytes, device, align=256):
    """(tensor, pointer aligned to `align`) of a device byte buffer of at least nbytes."""
    t = torch.empty(int(nbytes) + align, dtype=torch.uint8, device=device)
    return t, (t.data_ptr() + align - 1) // align * align


class Batch:
    """Many independent 2D lattices of one configuration (sizes (nx[i], ny[i])) advanced by one
    cooperative launch per composite step; pools and workspace are torch CUDA tensors."""

    def __init__(self, cfg, sizes, stream=None, device=None):
        import torch
        self.torch = torch
        self.cfg = cfg
        self.shapes = [(int(ny), int(nx)) for nx, ny in sizes]
        self.count = len(self.shapes)
        self._nx = (ctypes.c_int64 * self.count)(*[s[1] for s in self.shapes])
        self._ny = (ctypes.c_int64 * self.count)(*[s[0] for s in self.shapes])
        bs = BatchSizes()
        st = lib().eslbm_batch_query(ctypes.byref(cfg), self.count, self._nx, self._ny, ctypes.byref(bs))
        if st != OK:
            raise EslbmError(st, lib().eslbm_status_string(st).decode())
        self.sizes = bs
        self.device = torch.device(device or "cuda")
        self._pa, pa = _aligned(torch, bs.pool_bytes, self.device)
        self._pb, pb = _aligned(torch, bs.pool_bytes, self.device)
        self._ws, ws = _aligned(torch, bs.workspace_bytes, self.device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        h = ctypes.c_void_p()
        st = lib().eslbm_batch_create(ctypes.byref(cfg), self.count, self._nx, self._ny, pa, pb, ws,
                                      self.stream.cuda_stream, ctypes.byref(h))
        if st != OK:
            raise EslbmError(st, lib().eslbm_status_string(st).decode())
        self.h = h

    @property
    def M(self):
        return int(self.sizes.M)

    @property
    def total_cells(self):
        return int(self.sizes.total_cells)

    def _check(self, st):
        if st in (OK, WARN_OMEGA_FALLBACK):
            return st
        msg = lib().eslbm_status_string(st).decode()
        if getattr(self, "h", None) is not None:
            msg += ": " + lib().eslbm_batch_last_error(self.h).decode()
        raise EslbmError(st, msg)

    def close(self):
        if getattr(self, "h", None) is not None:
            lib().eslbm_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def pack(self, fields):
        """One flat float64 CUDA tensor from per-instance (M, ny, nx) fields."""
        torch = self.torch
        return torch.cat([torch.as_tensor(f, dtype=torch.float64).to(self.device).reshape(-1) for f in fields])

    def unpack(self, flat):
        """Per-instance (M, ny, nx) views of a flat tensor."""
        out, o = [], 0
        for ny, nx in self.shapes:
            n = self.M * ny * nx
            out.append(flat[o:o + n].reshape(self.M, ny, nx))
            o += n
        return out

    def init_equilibrium(self, fields):
        flat = fields if isinstance(fields, self.torch.Tensor) and fields.dim() == 1 else self.pack(fields)
        flat = flat.to(device=self.device, dtype=self.torch.float64).contiguous()
        return self._check(lib().eslbm_batch_init_equilibrium(self.h, flat.data_ptr(), 1))

    def step(self, n=1):
        return self._check(lib().eslbm_batch_step(self.h, int(n)))

    def moments_flat(self, out=None):
        t = out if out is not None else self.torch.empty(self.M * self.total_cells, dtype=self.torch.float64,
                                                         device=self.device)
        self._check(lib().eslbm_batch_read_moments(self.h, t.data_ptr(), 1))
        return t

    def moments(self):
        return self.unpack(self.moments_flat())

    def set_schedule(self, segment, blocks_per_sm, order):
        return self._check(lib().eslbm_batch_set_schedule(self.h, int(segment), int(blocks_per_sm), int(order)))

    def schedule(self):
        seg, bps, order = ctypes.c_int64(), ctypes.c_int32(), ctypes.c_int32()
        self._check(lib().eslbm_batch_get_schedule(self.h, ctypes.byref(seg), ctypes.byref(bps), ctypes.byref(order)))
        return int(seg.value), int(bps.value), int(order.value)

    def tune(self, steps=2):
        keep, p = _aligned(self.torch, self.sizes.pool_bytes, self.device)
        self._check(lib().eslbm_batch_tune(self.h, p, int(self.sizes.pool_bytes), int(steps)))
        return self.schedule()

    def use_graph(self, enable=True):
        return self._check(lib().eslbm_batch_use_graph(self.h, 1 if enable else 0))

    def diagnostics(self):
        d = Diagnostics()
        st = lib().eslbm_batch_get_diagnostics(self.h, ctypes.byref(d))
        self._check(st)
        return {"fallbacks": d.fallbacks, "entropy_increases": d.entropy_increases, "omega_min": d.omega_min,
                "omega_max": d.omega_max, "entropy_excess_max": d.entropy_excess_max, "status": st}

    def gradient(self, u0, dJ_duT, n, K=50):
        """Per-instance dJ/du0 (flat float64 CUDA tensor; inputs flat or per-instance lists)."""
        torch = self.torch
        nb = ctypes.c_uint64()
        self._check(lib().eslbm_batch_gradient_workspace(ctypes.byref(self.cfg), self.count, self._nx, self._ny,
                                                         int(n), int(K), ctypes.byref(nb)))
        keep, ws = _aligned(torch, nb.value, self.device)
        flat = lambda x: (x if isinstance(x, torch.Tensor) and x.dim() == 1 else self.pack(x)).to(
            device=self.device, dtype=torch.float64).contiguous()
        u0, g = flat(u0), flat(dJ_duT)
        out = torch.empty_like(u0)
        self._check(lib().eslbm_batch_gradient(self.h, u0.data_ptr(), g.data_ptr(), out.data_ptr(), int(n), int(K),
                                               ws, nb.value))
        return out
