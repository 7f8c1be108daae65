"""ctypes wrapper of the FP64 CPU oracle ``libqnsch_ref.so`` (test infrastructure).

Array layouts (numpy, C order, no ghost cells), as in ``qnsch_ref.h``:
    c, mu, p : (m2, m1)      cell centres
    u        : (m2, m1 + 1)  u_{i+1/2, j}, i = 0..m1
    v        : (m2 + 1, m1)  v_{i, j+1/2}, j = 0..m2
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "qnsch_ref.c")
_LIB = os.path.join(_HERE, "libqnsch_ref.so")

_D = ctypes.POINTER(ctypes.c_double)


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (-O2, no fast-math, no FMA contraction)."""
    hdr = os.path.join(_HERE, "qnsch_ref.h")
    stale = (not os.path.exists(_LIB) or
             os.path.getmtime(_LIB) < max(os.path.getmtime(_SRC), os.path.getmtime(hdr)))
    if force or stale:
        tmp = _LIB + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-std=c99", "-fPIC", "-shared", "-ffp-contract=off",
                               "-fno-fast-math", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        L = ctypes.CDLL(build())
        i, d, p, vp = ctypes.c_int, ctypes.c_double, _D, ctypes.c_void_p
        L.qnsch_ref_create.argtypes = [i, i, d, i, i, d, d, d, d, d, d, d, d, d,
                                       ctypes.POINTER(vp)]
        L.qnsch_ref_destroy.argtypes = [vp]
        L.qnsch_ref_set_option.argtypes = [vp, ctypes.c_char_p, d]
        L.qnsch_ref_get_option.argtypes = [vp, ctypes.c_char_p, p]
        L.qnsch_ref_levels.argtypes = [vp]
        L.qnsch_ref_ncolours_vanka.argtypes = [vp]
        for name in ("set_fields", "set_iterate"):
            getattr(L, "qnsch_ref_" + name).argtypes = [vp, p, p, p, p, p]
        for name in ("get_fields", "get_iterate"):
            getattr(L, "qnsch_ref_" + name).argtypes = [vp, p, p, p, p, p]
        L.qnsch_ref_get_history.argtypes = [vp, i, p, p, p, p, p, p]
        L.qnsch_ref_set_history.argtypes = [vp, i, d, p, p, p, p, p]
        L.qnsch_ref_step.argtypes = [vp, d, ctypes.POINTER(i), p]
        L.qnsch_ref_begin_step.argtypes = [vp, d]
        L.qnsch_ref_vcycle.argtypes = [vp, p]
        L.qnsch_ref_commit_step.argtypes = [vp]
        L.qnsch_ref_residual.argtypes = [vp, p, p, p, p, p, p]
        L.qnsch_ref_smooth_ch.argtypes = [vp, i]
        L.qnsch_ref_smooth_vanka.argtypes = [vp, i]
        L.qnsch_ref_smooth.argtypes = [vp, i]
        L.qnsch_ref_ch_jacobian.argtypes = [vp, i, i, p, p]
        L.qnsch_ref_vanka_jacobian.argtypes = [vp, i, i, p, p, ctypes.POINTER(i)]
        L.qnsch_ref_mass.argtypes = [vp, p, p]
        L.qnsch_ref_energy.argtypes = [vp, p]
        L.qnsch_ref_iterate_energy.argtypes = [vp, p]
        L.qnsch_ref_iterate_dissipation.argtypes = [vp, p]
        L.qnsch_ref_params.argtypes = [vp, p]
        L.qnsch_ref_secants.argtypes = [vp, d, d, p]
        L.qnsch_ref_transfer.argtypes = [vp, i, i, p, p]
        L.qnsch_ref_diagnostics.argtypes = [vp, p]
        L.qnsch_ref_projected_velocity.argtypes = [vp, p, p]
        L.qnsch_ref_divergence.argtypes = [vp, p]
        _lib = L
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(_D)


class RefError(RuntimeError):
    pass


def _check(rc, what):
    if rc != 0:
        raise RefError("%s failed with status %d" % (what, rc))


class RefSolver:
    """One q-NSCH instance in the oracle."""

    def __init__(self, m1, m2, Lx=1.0, periodic_x=False, levels=0, rho1=1.0, rho2=1.0,
                 eta1=1.0, eta2=1.0, Re=100.0, We=10.0, Pe=100.0, Cn=0.01, Fr=math.inf,
                 **options):
        self.m1, self.m2 = int(m1), int(m2)
        self.h = Lx / m1
        self.periodic_x = bool(periodic_x)
        h = ctypes.c_void_p()
        _check(lib().qnsch_ref_create(self.m1, self.m2, Lx, int(periodic_x), int(levels), rho1,
                                      rho2, eta1, eta2, Re, We, Pe, Cn, Fr, ctypes.byref(h)),
               "qnsch_ref_create")
        self._h = h
        for k, v in options.items():
            self.set_option(k, v)

    def close(self):
        if self._h is not None and self._h.value:
            lib().qnsch_ref_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ---- shapes ----
    def shapes(self):
        m1, m2 = self.m1, self.m2
        return dict(c=(m2, m1), mu=(m2, m1), p=(m2, m1), u=(m2, m1 + 1), v=(m2 + 1, m1))

    def zeros(self):
        return {k: np.zeros(s) for k, s in self.shapes().items()}

    # ---- options ----
    def set_option(self, key, value):
        _check(lib().qnsch_ref_set_option(self._h, key.encode(), float(value)), "set_option " + key)

    def get_option(self, key):
        out = ctypes.c_double()
        _check(lib().qnsch_ref_get_option(self._h, key.encode(), ctypes.byref(out)), "get_option")
        return out.value

    @property
    def levels(self):
        return lib().qnsch_ref_levels(self._h)

    @property
    def ncolours_vanka(self):
        return lib().qnsch_ref_ncolours_vanka(self._h)

    def params(self):
        out = np.zeros(8)
        _check(lib().qnsch_ref_params(self._h, _ptr(out)), "params")
        keys = ("alpha", "eta", "K", "Lam", "M", "Fr_inv", "eps_m", "h")
        return dict(zip(keys, out.tolist()))

    def transfer(self, level, op, a, out_shape):
        """qnsch_ref_transfer: op 0-2 restrict fine cells / x-edges / y-edges of
        level `level` to level + 1, op 3-5 prolongate from level + 1."""
        a = np.ascontiguousarray(a, dtype=np.float64)
        out = np.zeros(out_shape)
        _check(lib().qnsch_ref_transfer(self._h, int(level), int(op), _ptr(a), _ptr(out)),
               "transfer")
        return out

    def secants(self, a, b):
        """F(a), F(b), g(a,b), dg/da(a,b), rho(a), rho(b), r(a,b) (Secs. 2.1, 4.1)."""
        out = np.zeros(7)
        _check(lib().qnsch_ref_secants(self._h, float(a), float(b), _ptr(out)), "secants")
        keys = ("Fa", "Fb", "g", "g_a", "rho_a", "rho_b", "r")
        return dict(zip(keys, out.tolist()))

    # ---- fields ----
    def _in(self, f):
        out = {}
        for k, s in self.shapes().items():
            a = np.ascontiguousarray(f[k], dtype=np.float64)
            if a.shape != s:
                raise ValueError("%s has shape %s, expected %s" % (k, a.shape, s))
            out[k] = a
        return out

    def set_fields(self, f):
        a = self._in(f)
        _check(lib().qnsch_ref_set_fields(self._h, _ptr(a["c"]), _ptr(a["mu"]), _ptr(a["u"]),
                                          _ptr(a["v"]), _ptr(a["p"])), "set_fields")

    def get_fields(self):
        a = self.zeros()
        _check(lib().qnsch_ref_get_fields(self._h, _ptr(a["c"]), _ptr(a["mu"]), _ptr(a["u"]),
                                          _ptr(a["v"]), _ptr(a["p"])), "get_fields")
        return a

    def history(self, k):
        """(fields, dt) of the k-th state committed before the current one."""
        a = self.zeros()
        dt = np.zeros(1)
        _check(lib().qnsch_ref_get_history(self._h, int(k), _ptr(dt), _ptr(a["c"]), _ptr(a["mu"]),
                                           _ptr(a["u"]), _ptr(a["v"]), _ptr(a["p"])),
               "get_history")
        return a, float(dt[0])

    def set_history(self, k, f, dt):
        a = self._in(f)
        _check(lib().qnsch_ref_set_history(self._h, int(k), float(dt), _ptr(a["c"]), _ptr(a["mu"]),
                                           _ptr(a["u"]), _ptr(a["v"]), _ptr(a["p"])),
               "set_history")

    def set_iterate(self, f):
        a = self._in(f)
        _check(lib().qnsch_ref_set_iterate(self._h, _ptr(a["c"]), _ptr(a["mu"]), _ptr(a["u"]),
                                           _ptr(a["v"]), _ptr(a["p"])), "set_iterate")

    def get_iterate(self):
        a = self.zeros()
        _check(lib().qnsch_ref_get_iterate(self._h, _ptr(a["c"]), _ptr(a["mu"]), _ptr(a["u"]),
                                           _ptr(a["v"]), _ptr(a["p"])), "get_iterate")
        return a

    # ---- stepping ----
    def step(self, dt):
        n = ctypes.c_int()
        r = ctypes.c_double()
        rc = lib().qnsch_ref_step(self._h, float(dt), ctypes.byref(n), ctypes.byref(r))
        _check(rc, "step")
        return n.value, r.value

    def begin_step(self, dt):
        _check(lib().qnsch_ref_begin_step(self._h, float(dt)), "begin_step")

    def vcycle(self):
        out = np.zeros(10)
        _check(lib().qnsch_ref_vcycle(self._h, _ptr(out)), "vcycle")
        return out

    def commit_step(self):
        _check(lib().qnsch_ref_commit_step(self._h), "commit_step")

    def residual(self):
        r = self.zeros()
        n = np.zeros(10)
        _check(lib().qnsch_ref_residual(self._h, _ptr(r["c"]), _ptr(r["mu"]), _ptr(r["p"]),
                                        _ptr(r["u"]), _ptr(r["v"]), _ptr(n)), "residual")
        return r, n

    def smooth_ch(self, colour):
        _check(lib().qnsch_ref_smooth_ch(self._h, int(colour)), "smooth_ch")

    def smooth_vanka(self, colour):
        _check(lib().qnsch_ref_smooth_vanka(self._h, int(colour)), "smooth_vanka")

    def smooth(self, sweeps=1):
        _check(lib().qnsch_ref_smooth(self._h, int(sweeps)), "smooth")

    def ch_jacobian(self, i, j):
        J = np.zeros(4)
        R = np.zeros(2)
        _check(lib().qnsch_ref_ch_jacobian(self._h, i, j, _ptr(J), _ptr(R)), "ch_jacobian")
        return J.reshape(2, 2), R

    def vanka_jacobian(self, i, j):
        J = np.zeros(25)
        R = np.zeros(5)
        act = (ctypes.c_int * 5)()
        _check(lib().qnsch_ref_vanka_jacobian(self._h, i, j, _ptr(J), _ptr(R), act),
               "vanka_jacobian")
        return J.reshape(5, 5), R, np.array(list(act), dtype=bool)

    # ---- diagnostics ----
    def mass(self):
        a, b = ctypes.c_double(), ctypes.c_double()
        _check(lib().qnsch_ref_mass(self._h, ctypes.byref(a), ctypes.byref(b)), "mass")
        return a.value, b.value

    def energy(self):
        e = ctypes.c_double()
        _check(lib().qnsch_ref_energy(self._h, ctypes.byref(e)), "energy")
        return e.value

    DIAG_KEYS = ("Vc", "yc", "div_max", "div_l2", "div_expansion", "div_compression", "a1",
                 "y_top", "y_bottom")

    def diagnostics(self):
        """Sec. 8 diagnostics of the committed state (rise velocity, centroid,
        divergence extremes and l2 norm, capillary amplitude, interface tips)."""
        out = np.zeros(9)
        _check(lib().qnsch_ref_diagnostics(self._h, _ptr(out)), "diagnostics")
        return dict(zip(self.DIAG_KEYS, out.tolist()))

    def projected_velocity(self):
        """Projection method: u^{n+1}, v^{n+1} of the pending iterate."""
        a = self.zeros()
        _check(lib().qnsch_ref_projected_velocity(self._h, _ptr(a["u"]), _ptr(a["v"])),
               "projected_velocity")
        return a["u"], a["v"]

    def divergence(self):
        """d_x u + d_y v of the committed state, shape (m2, m1)."""
        out = np.zeros((self.m2, self.m1))
        _check(lib().qnsch_ref_divergence(self._h, _ptr(out)), "divergence")
        return out

    def iterate_energy(self):
        e = ctypes.c_double()
        _check(lib().qnsch_ref_iterate_energy(self._h, ctypes.byref(e)), "iterate_energy")
        return e.value

    def iterate_dissipation(self):
        e = ctypes.c_double()
        _check(lib().qnsch_ref_iterate_dissipation(self._h, ctypes.byref(e)),
               "iterate_dissipation")
        return e.value
