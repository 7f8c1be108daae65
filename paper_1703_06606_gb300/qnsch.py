"""Thin ctypes binding of libqnsch.so (include/qnsch.h): argument marshalling only.

Every numerical step runs in the CUDA kernels of the library.  There is no CPU
fallback: if the library cannot be loaded, or no GPU is present, calls raise.

Array layouts (numpy / torch, C order, float64, no ghost cells):
    c, mu, p : (m2, m1); u : (m2, m1 + 1); v : (m2 + 1, m1)
"""
from __future__ import annotations

import ctypes
import math
import os

import numpy as np

from . import build as _build

_D = ctypes.POINTER(ctypes.c_double)
_VP = ctypes.c_void_p

STATUS = {0: "OK", -1: "EINVAL", -2: "ENODEV", -3: "ENOMEM", -4: "ENOTCONV", -5: "ENAN",
          -6: "ETIMEOUT", -7: "EBUDGET", -8: "ESTATE", -9: "ECUDA"}


class QnschError(RuntimeError):
    def __init__(self, what, code):
        super().__init__("%s failed: QNSCH_%s (%d)" % (what, STATUS.get(code, "?"), code))
        self.code = code


class _Grid(ctypes.Structure):
    _fields_ = [("m1", ctypes.c_int), ("m2", ctypes.c_int), ("Lx", ctypes.c_double),
                ("periodic_x", ctypes.c_int), ("periodic_y", ctypes.c_int),
                ("levels", ctypes.c_int)]


_lib = None


def lib():
    """Load (building first if stale) the in-tree libqnsch.so."""
    global _lib
    if _lib is None:
        path = _build.LIB
        if not os.path.exists(path) or _build.is_stale():
            path = _build.build()
        L = ctypes.CDLL(path)
        i, d, p = ctypes.c_int, ctypes.c_double, _D
        L.qnsch_create.argtypes = [ctypes.POINTER(_Grid), d, d, d, d, d, d, d, d, d,
                                   ctypes.POINTER(_VP)]
        L.qnsch_destroy.argtypes = [_VP]
        L.qnsch_set_option.argtypes = [_VP, ctypes.c_char_p, d]
        L.qnsch_get_option.argtypes = [_VP, ctypes.c_char_p, p]
        L.qnsch_set_stream.argtypes = [_VP, _VP]
        L.qnsch_levels.argtypes = [_VP]
        L.qnsch_ncolours_vanka.argtypes = [_VP]
        for name in ("set_fields", "get_fields", "set_fields_device", "get_fields_device",
                     "set_iterate", "get_iterate"):
            getattr(L, "qnsch_" + name).argtypes = [_VP, _VP, _VP, _VP, _VP, _VP]
        L.qnsch_get_history.argtypes = [_VP, i, p, _VP, _VP, _VP, _VP, _VP]
        L.qnsch_set_history.argtypes = [_VP, i, d, _VP, _VP, _VP, _VP, _VP]
        L.qnsch_step.argtypes = [_VP, d, ctypes.POINTER(i), p]
        L.qnsch_step_launch.argtypes = [_VP, d]
        L.qnsch_step_poll.argtypes = [_VP, ctypes.POINTER(i), ctypes.POINTER(i), p,
                                      ctypes.POINTER(i), p]
        L.qnsch_begin_step.argtypes = [_VP, d]
        L.qnsch_vcycle.argtypes = [_VP, p]
        L.qnsch_commit_step.argtypes = [_VP]
        L.qnsch_mass.argtypes = [_VP, p, p]
        L.qnsch_diagnostics.argtypes = [_VP, p]
        L.qnsch_divergence.argtypes = [_VP, p]
        L.qnsch_energy.argtypes = [_VP, p, p]
        L.qnsch_iterate_energy.argtypes = [_VP, p, p]
        L.qnsch_residual.argtypes = [_VP, _VP, _VP, _VP, _VP, _VP, p]
        L.qnsch_smooth_ch.argtypes = [_VP, i]
        L.qnsch_smooth_vanka.argtypes = [_VP, i]
        L.qnsch_smooth.argtypes = [_VP, i]
        L.qnsch_set_allocator.argtypes = [_VP, _VP, _VP]
        L.qnsch_profile.argtypes = [_VP, i]
        L.qnsch_profile_read.argtypes = [_VP, ctypes.POINTER(ctypes.c_longlong), p]
        L.qnsch_profile_read_kind.argtypes = [_VP, i, ctypes.POINTER(ctypes.c_longlong), p, p]
        L.qnsch_kernel_launches.argtypes = [ctypes.POINTER(ctypes.c_longlong)]
        L.qnsch_set_budget.argtypes = [ctypes.c_size_t]
        L.qnsch_version.argtypes = [ctypes.POINTER(i)] * 3
        L.qnsch_budget.argtypes = [ctypes.POINTER(ctypes.c_size_t), ctypes.POINTER(ctypes.c_size_t)]
        L.qnsch_mass_noalloc.argtypes = [_VP, i, i, d, d, d, _VP, _VP]
        L.qnsch_batch_create.argtypes = [i, ctypes.POINTER(_VP), ctypes.POINTER(_VP)]
        L.qnsch_batch_step.argtypes = [_VP, p, ctypes.POINTER(i), ctypes.POINTER(i)]
        L.qnsch_batch_size.argtypes = [_VP]
        L.qnsch_batch_set_option.argtypes = [_VP, ctypes.c_char_p, d]
        L.qnsch_batch_step_times.argtypes = [_VP, p]
        L.qnsch_batch_destroy.argtypes = [_VP]
        L.qnsch_footprint.argtypes = [ctypes.POINTER(_Grid), i, ctypes.POINTER(ctypes.c_size_t)]
        _lib = L
    return _lib


def kernel_launches():
    """Kernels issued by libqnsch.so in this process (host-side count)."""
    n = ctypes.c_longlong()
    _check(lib().qnsch_kernel_launches(ctypes.byref(n)), "qnsch_kernel_launches")
    return n.value


def version():
    """qnsch_version: (major, minor, patch) of the loaded library."""
    v = [ctypes.c_int() for _ in range(3)]
    _check(lib().qnsch_version(*[ctypes.byref(x) for x in v]), "qnsch_version")
    return tuple(x.value for x in v)


def set_budget(nbytes):
    """qnsch_set_budget: the process's device-memory budget in bytes (0: none)."""
    _check(lib().qnsch_set_budget(int(nbytes)), "qnsch_set_budget")


def budget():
    """qnsch_budget: (budget in bytes, bytes reserved by live handles)."""
    b, u = ctypes.c_size_t(), ctypes.c_size_t()
    _check(lib().qnsch_budget(ctypes.byref(b), ctypes.byref(u)), "qnsch_budget")
    return b.value, u.value


def mass_noalloc(c, h, rho1, rho2, out2, stream=None):
    """qnsch_mass_noalloc: h^2 sum rho(c), h^2 sum rho(c) c of a caller-owned CUDA
    float64 tensor c (m2, m1) into the caller-owned CUDA float64 tensor out2 (2,),
    queued on `stream` (torch stream or handle) without allocating anything.  The
    caller synchronises before reading out2."""
    if not (c.is_cuda and c.is_contiguous() and c.dim() == 2 and out2.is_cuda and
            out2.numel() >= 2):
        raise ValueError("need a contiguous 2-D CUDA tensor c and a CUDA tensor out2 of 2")
    handle = getattr(stream, "cuda_stream", stream)
    m2, m1 = c.shape
    _check(lib().qnsch_mass_noalloc(c.data_ptr(), int(m1), int(m2), float(h), float(rho1),
                                    float(rho2), out2.data_ptr(), handle or None),
           "qnsch_mass_noalloc")


def _check(rc, what):
    if rc != 0:
        raise QnschError(what, rc)


def _np_ptr(a):
    return None if a is None else a.ctypes.data


class Solver:
    """One q-NSCH instance on the GPU (the handle of qnsch_create)."""

    FIELDS = ("c", "mu", "u", "v", "p")  # argument order of the C calls

    def __init__(self, m1, m2, Lx=1.0, periodic_x=False, levels=0, rho1=1.0, rho2=1.0,
                 eta1=1.0, eta2=1.0, Re=100.0, We=10.0, Pe=100.0, Cn=0.01, Fr=math.inf,
                 stream=None, **options):
        self.m1, self.m2 = int(m1), int(m2)
        self.periodic_x = bool(periodic_x)
        self.h = Lx / m1
        # the creation parameters, as a checkpoint records them
        self.params = dict(m1=self.m1, m2=self.m2, Lx=float(Lx), periodic_x=self.periodic_x,
                           levels=int(levels), rho1=float(rho1), rho2=float(rho2),
                           eta1=float(eta1), eta2=float(eta2), Re=float(Re), We=float(We),
                           Pe=float(Pe), Cn=float(Cn), Fr=float(Fr))
        g = _Grid(self.m1, self.m2, float(Lx), int(periodic_x), 0, int(levels))
        h = _VP()
        _check(lib().qnsch_create(ctypes.byref(g), rho1, rho2, eta1, eta2, Re, We, Pe, Cn, Fr,
                                  ctypes.byref(h)), "qnsch_create")
        self._h = h
        if stream is not None:
            self.set_stream(stream)
        for k, v in options.items():
            self.set_option(k, v)

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            lib().qnsch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ---- configuration ----
    def set_stream(self, stream):
        """stream: a torch.cuda.Stream, an int handle, or None for the default stream."""
        handle = getattr(stream, "cuda_stream", stream)
        _check(lib().qnsch_set_stream(self._h, handle or None), "qnsch_set_stream")

    def set_option(self, key, value):
        _check(lib().qnsch_set_option(self._h, key.encode(), float(value)), "set_option " + key)

    def get_option(self, key):
        out = ctypes.c_double()
        _check(lib().qnsch_get_option(self._h, key.encode(), ctypes.byref(out)), "get_option")
        return out.value

    def options(self):
        """Every per-handle option (the keys a checkpoint records) -> value."""
        from . import checkpoint
        return {k: self.get_option(k) for k in checkpoint.OPTIONS}

    # ---- checkpoint / resume ----
    def save_checkpoint(self, path, t=0.0, n=0):
        """Write the committed state, creation parameters and options (plus the
        caller's time t and step count n) to the .npz file `path`, with the
        earlier states the option "predictor" extrapolates from."""
        from . import checkpoint
        hist = [self.history(k) for k in range(int(self.get_option("history")))]
        checkpoint.save(path, self.get_fields(), self.params, self.options(), t, n,
                        library=version(), history=hist)

    @classmethod
    def from_checkpoint(cls, path, stream=None, **overrides):
        """A new Solver in the state a checkpoint recorded: (solver, t, n).
        `overrides` replace recorded options (e.g. a different tol)."""
        from . import checkpoint
        fields, params, opts, t, n = checkpoint.load(path)
        s = cls(**params, stream=stream)
        for k, v in dict(opts, **overrides).items():
            s.set_option(k, v)
        s.set_fields(fields)
        for k, (hf, dt) in enumerate(checkpoint.load_history(path)):
            s.set_history(k, hf, dt)
        return s, t, n

    @property
    def levels(self):
        return lib().qnsch_levels(self._h)

    @property
    def ncolours_vanka(self):
        return lib().qnsch_ncolours_vanka(self._h)

    def shapes(self):
        m1, m2 = self.m1, self.m2
        return dict(c=(m2, m1), mu=(m2, m1), p=(m2, m1), u=(m2, m1 + 1), v=(m2 + 1, m1))

    def zeros(self):
        return {k: np.zeros(s) for k, s in self.shapes().items()}

    def _host_in(self, f):
        out = {}
        for k, s in self.shapes().items():
            a = np.ascontiguousarray(f[k], dtype=np.float64)
            if a.shape != s:
                raise ValueError("%s has shape %s, expected %s" % (k, a.shape, s))
            out[k] = a
        return out

    def _host_call(self, fn, f, what):
        a = self._host_in(f)
        _check(fn(self._h, *[_np_ptr(a[k]) for k in self.FIELDS]), what)

    def _host_get(self, fn, what):
        a = self.zeros()
        _check(fn(self._h, *[_np_ptr(a[k]) for k in self.FIELDS]), what)
        return a

    # ---- fields ----
    def set_fields(self, f):
        self._host_call(lib().qnsch_set_fields, f, "qnsch_set_fields")

    def get_fields(self):
        return self._host_get(lib().qnsch_get_fields, "qnsch_get_fields")

    def set_fields_device(self, t):
        """t: dict of contiguous float64 CUDA tensors in the host layouts."""
        ptrs = []
        for k in self.FIELDS:
            x = t[k]
            if tuple(x.shape) != self.shapes()[k] or not x.is_contiguous() or not x.is_cuda:
                raise ValueError("field %s: need a contiguous CUDA tensor of shape %s"
                                 % (k, self.shapes()[k]))
            ptrs.append(x.data_ptr())
        _check(lib().qnsch_set_fields_device(self._h, *ptrs), "qnsch_set_fields_device")

    def get_fields_device(self, t):
        ptrs = [t[k].data_ptr() for k in self.FIELDS]
        _check(lib().qnsch_get_fields_device(self._h, *ptrs), "qnsch_get_fields_device")

    def set_iterate(self, f):
        self._host_call(lib().qnsch_set_iterate, f, "qnsch_set_iterate")

    def history(self, k):
        """qnsch_get_history: (fields, dt) of the k-th state committed before the
        current one (0 the most recent)."""
        a = self.zeros()
        dt = ctypes.c_double()
        _check(lib().qnsch_get_history(self._h, int(k), ctypes.byref(dt),
                                       *[_np_ptr(a[q]) for q in self.FIELDS]),
               "qnsch_get_history")
        return a, dt.value

    def set_history(self, k, f, dt):
        """qnsch_set_history: the k-th earlier state and the step size that left it."""
        a = self._host_in(f)
        _check(lib().qnsch_set_history(self._h, int(k), float(dt),
                                       *[_np_ptr(a[q]) for q in self.FIELDS]),
               "qnsch_set_history")

    def get_iterate(self):
        return self._host_get(lib().qnsch_get_iterate, "qnsch_get_iterate")

    # ---- stepping ----
    def step(self, dt):
        n = ctypes.c_int()
        r = ctypes.c_double()
        _check(lib().qnsch_step(self._h, float(dt), ctypes.byref(n), ctypes.byref(r)),
               "qnsch_step")
        return n.value, r.value

    def step_launch(self, dt):
        """qnsch_step_launch: queue one whole step and return at once."""
        _check(lib().qnsch_step_launch(self._h, float(dt)), "qnsch_step_launch")

    def step_poll(self):
        """qnsch_step_poll: None while the launched step runs, else
        (n_vcycles, final_residual, status, device_ms); status is the code
        qnsch_step would have returned (0 on success)."""
        done, n, st = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        r, ms = ctypes.c_double(), ctypes.c_double()
        _check(lib().qnsch_step_poll(self._h, ctypes.byref(done), ctypes.byref(n),
                                     ctypes.byref(r), ctypes.byref(st), ctypes.byref(ms)),
               "qnsch_step_poll")
        if not done.value:
            return None
        return n.value, r.value, st.value, ms.value

    def begin_step(self, dt):
        _check(lib().qnsch_begin_step(self._h, float(dt)), "qnsch_begin_step")

    def vcycle(self):
        out = np.zeros(10)
        _check(lib().qnsch_vcycle(self._h, out.ctypes.data_as(_D)), "qnsch_vcycle")
        return out

    def commit_step(self):
        _check(lib().qnsch_commit_step(self._h), "qnsch_commit_step")

    def residual(self):
        r = self.zeros()
        n = np.zeros(10)
        _check(lib().qnsch_residual(self._h, _np_ptr(r["c"]), _np_ptr(r["mu"]), _np_ptr(r["p"]),
                                    _np_ptr(r["u"]), _np_ptr(r["v"]), n.ctypes.data_as(_D)),
               "qnsch_residual")
        return r, n

    def smooth_ch(self, colour):
        _check(lib().qnsch_smooth_ch(self._h, int(colour)), "qnsch_smooth_ch")

    def smooth_vanka(self, colour):
        _check(lib().qnsch_smooth_vanka(self._h, int(colour)), "qnsch_smooth_vanka")

    def smooth(self, sweeps=1):
        _check(lib().qnsch_smooth(self._h, int(sweeps)), "qnsch_smooth")

    # ---- measurement ----
    # kinds of timed launches (qnsch_profile's bits)
    PROFILE_KINDS = ("vanka_finest", "vanka_levels", "coarse_vcycle", "ch", "wave", "skew")

    def profile(self, enable=True):
        """enable: True (the finest-level Vanka launches), False, or a bit mask
        over PROFILE_KINDS."""
        mask = int(enable) if not isinstance(enable, bool) else int(enable)
        _check(lib().qnsch_profile(self._h, mask), "qnsch_profile")

    def profile_read_kind(self, kind):
        """(launches, total ms, cell visits) of one kind of timed launch."""
        k = self.PROFILE_KINDS.index(kind) if isinstance(kind, str) else int(kind)
        n, ms, vis = ctypes.c_longlong(), ctypes.c_double(), ctypes.c_double()
        _check(lib().qnsch_profile_read_kind(self._h, k, ctypes.byref(n), ctypes.byref(ms),
                                             ctypes.byref(vis)), "qnsch_profile_read_kind")
        return n.value, ms.value, vis.value

    def profile_read(self):
        n, ms = ctypes.c_longlong(), ctypes.c_double()
        _check(lib().qnsch_profile_read(self._h, ctypes.byref(n), ctypes.byref(ms)),
               "qnsch_profile_read")
        return n.value, ms.value

    # ---- diagnostics ----
    def mass(self):
        a, b = ctypes.c_double(), ctypes.c_double()
        _check(lib().qnsch_mass(self._h, ctypes.byref(a), ctypes.byref(b)), "qnsch_mass")
        return a.value, b.value

    def energy(self):
        e, d = ctypes.c_double(), ctypes.c_double()
        _check(lib().qnsch_energy(self._h, ctypes.byref(e), ctypes.byref(d)), "qnsch_energy")
        return e.value, d.value

    DIAG_KEYS = ("Vc", "yc", "div_max", "div_l2", "div_expansion", "div_compression", "a1",
                 "y_top", "y_bottom")

    def diagnostics(self):
        """qnsch_diagnostics: Sec. 8 diagnostics of the committed state as a dict."""
        out = np.zeros(9)
        _check(lib().qnsch_diagnostics(self._h, out.ctypes.data_as(ctypes.POINTER(ctypes.c_double))),
               "qnsch_diagnostics")
        return dict(zip(self.DIAG_KEYS, out.tolist()))

    def divergence(self):
        """qnsch_divergence: d_x u + d_y v of the committed state, shape (m2, m1)."""
        out = np.zeros((self.m2, self.m1))
        _check(lib().qnsch_divergence(self._h, out.ctypes.data_as(ctypes.POINTER(ctypes.c_double))),
               "qnsch_divergence")
        return out

    def iterate_energy(self):
        e, d = ctypes.c_double(), ctypes.c_double()
        _check(lib().qnsch_iterate_energy(self._h, ctypes.byref(e), ctypes.byref(d)),
               "qnsch_iterate_energy")
        return e.value, d.value


def footprint(m1, m2, periodic_x=False, levels=0, precision=0, Lx=1.0):
    """Device bytes of one handle (qnsch_footprint), computed without allocating."""
    g = _Grid(int(m1), int(m2), float(Lx), int(periodic_x), 0, int(levels))
    out = ctypes.c_size_t()
    _check(lib().qnsch_footprint(ctypes.byref(g), int(precision), ctypes.byref(out)),
           "qnsch_footprint")
    return out.value


class Batch:
    """qnsch_batch_*: step several Solver instances together (their kernels run
    concurrently on the GPU); each instance keeps its own tolerance and result."""

    def __init__(self, solvers, max_inflight=0):
        self.solvers = list(solvers)
        arr = (_VP * len(self.solvers))(*[sv._h.value for sv in self.solvers])
        h = _VP()
        _check(lib().qnsch_batch_create(len(self.solvers), arr, ctypes.byref(h)),
               "qnsch_batch_create")
        self._h = h
        if max_inflight:
            self.set_option("max_inflight", max_inflight)

    def step_times(self):
        """qnsch_batch_step_times: each member's device span (ms) in the last step."""
        out = np.zeros(len(self.solvers))
        _check(lib().qnsch_batch_step_times(self._h, out.ctypes.data_as(_D)),
               "qnsch_batch_step_times")
        return out

    def set_option(self, key, value):
        """qnsch_batch_set_option ("max_inflight": members stepping at once, 0 = all)."""
        _check(lib().qnsch_batch_set_option(self._h, key.encode(), float(value)),
               "qnsch_batch_set_option " + key)

    def step(self, dt):
        n = len(self.solvers)
        dts = np.ascontiguousarray(np.broadcast_to(np.asarray(dt, dtype=np.float64), (n,)))
        st = (ctypes.c_int * n)()
        cy = (ctypes.c_int * n)()
        _check(lib().qnsch_batch_step(self._h, dts.ctypes.data_as(_D), st, cy), "qnsch_batch_step")
        return list(st), list(cy)

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            lib().qnsch_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
