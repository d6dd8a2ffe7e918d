"""ctypes wrapper of the plain scalar FP64 CPU oracle (oracle/fdf_oracle.c).

TEST INFRASTRUCTURE ONLY: imported by tests/, by ``__graft_entry__.smoke()``
and by the CPU-baseline leg of bench.py.  The product package never imports
it.  Inputs (parameters, transfer tables, the Fermi-Dirac CDF table) are passed
in by the caller; the oracle shares no code with the CUDA path.
"""
import ctypes as C
import os

import numpy as np

from . import build as _build

_lib = None


class OrParams(C.Structure):
    _fields_ = [
        ("box", C.c_double),
        ("n_part", C.c_int64),
        ("n_grid", C.c_int32),
        ("n_species", C.c_int32),
        ("m_ev", C.c_double * 4),
        ("T_K", C.c_double),
        ("z_start", C.c_double),
        ("z_end", C.c_double),
        ("n_steps", C.c_int32),
        ("flags", C.c_int32),
        ("seed", C.c_uint64),
        ("h", C.c_double),
        ("omega_m", C.c_double),
        ("omega_r", C.c_double),
        ("A_s", C.c_double),
        ("n_s", C.c_double),
        ("k_pivot", C.c_double),
        ("interp_order", C.c_int32),
        ("superstep_tol", C.c_double),
        ("eom", C.c_int32),
    ]


class OrTables(C.Structure):
    _fields_ = [
        ("nk", C.c_int32),
        ("na", C.c_int32),
        ("lnk", C.POINTER(C.c_double)),
        ("lna", C.POINTER(C.c_double)),
        ("T_psi", C.POINTER(C.c_double)),
        ("T_phi", C.POINTER(C.c_double)),
        ("dTphi_dlna", C.POINTER(C.c_double)),
        ("ncdf", C.c_int32),
        ("cdf_t", C.POINTER(C.c_double)),
        ("cdf_F", C.POINTER(C.c_double)),
    ]


_D = C.POINTER(C.c_double)
_U32 = C.POINTER(C.c_uint32)
_I64 = C.POINTER(C.c_int64)


def lib():
    """Load liboracle.so, building it first if needed."""
    global _lib
    if _lib is None:
        path = _build.build()
        L = C.CDLL(path)
        L.or_philox4x32_10.argtypes = [_U32, _U32, _U32]
        L.or_hubble.argtypes = [C.POINTER(OrParams), C.c_double]
        L.or_hubble.restype = C.c_double
        L.or_gauss_legendre.argtypes = [C.c_int, _D, _D]
        L.or_dtau.argtypes = [C.POINTER(OrParams), C.c_double, C.c_double]
        L.or_dtau.restype = C.c_double
        L.or_eps_integral.argtypes = [C.POINTER(OrParams), C.c_double, C.c_double, C.c_double, C.c_double,
                                      C.c_int]
        L.or_eps_integral.restype = C.c_double
        L.or_tau.argtypes = [C.POINTER(OrParams), C.c_double]
        L.or_tau.restype = C.c_double
        L.or_temperature_ev.argtypes = [C.POINTER(OrParams)]
        L.or_temperature_ev.restype = C.c_double
        L.or_fd_cdf.argtypes = [C.c_double]
        L.or_fd_cdf.restype = C.c_double
        L.or_sample.argtypes = [C.POINTER(OrParams), C.POINTER(OrTables), _I64, C.c_int64, _U32, _D, _D]
        L.or_fd_inverse.argtypes = [C.POINTER(OrTables), C.c_double]
        L.or_fd_inverse.restype = C.c_double
        L.or_noise.argtypes = [C.POINTER(OrParams), _D]
        L.or_interp_table.argtypes = [C.POINTER(OrTables), _D, C.c_double, C.c_double]
        L.or_interp_table.restype = C.c_double
        L.or_supersteps.argtypes = [C.POINTER(OrParams), C.POINTER(OrTables), C.POINTER(C.c_int32)]
        L.or_tf_change.argtypes = [C.POINTER(OrParams), C.POINTER(OrTables), C.c_int, C.c_int]
        L.or_tf_change.restype = C.c_double
        L.or_fft3d_inverse.argtypes = [C.c_int, _D]
        L.or_dft3d_inverse_naive.argtypes = [C.c_int, _D, _D]
        L.or_fields.argtypes = [C.POINTER(OrParams), C.POINTER(OrTables), _D, C.c_double, C.c_uint, _D, _D]
        L.or_gather.argtypes = [C.POINTER(OrParams), _D, _D, _D]
        L.or_initial.argtypes = [C.POINTER(OrParams), C.POINTER(OrTables), _D, _I64, C.c_int64, _U32, _D, _D,
                                 _D, _D, _D]
        L.or_integrate.argtypes = [C.POINTER(OrParams), C.POINTER(OrTables), _D, _I64, C.c_int64, C.c_int,
                                   C.c_int, _D, _D, _D]
        L.or_weights.argtypes = [C.POINTER(OrParams), C.c_int64, _D, _D, _D]
        L.or_accel_terms.argtypes = [C.POINTER(OrParams), C.POINTER(OrTables), _D, _I64, C.c_int64, C.c_int,
                                     _D, _D, _D]
        L.or_deposit.argtypes = [C.POINTER(OrParams), _I64, C.c_int64, _D, _D, _D, C.c_double, C.c_int, _D]
        L.or_lna.argtypes = [C.POINTER(OrParams), C.c_double]
        L.or_lna.restype = C.c_double
        L.or_num_threads.restype = C.c_int
        _lib = L
    return _lib


def _p(a, ct):
    return a.ctypes.data_as(C.POINTER(ct))


class Oracle:
    """The oracle for one parameter set and one set of input tables.

    ``params`` is a dict with the keys of OrParams (m_ev a list of up to 4);
    ``tables`` a dict with lnk, lna, T_psi, T_phi, dTphi_dlna ([na][nk]),
    cdf_t and cdf_F (numpy float64 arrays).
    """

    def __init__(self, params, tables):
        self.params = dict(params)
        P = OrParams()
        for k, v in self.params.items():
            if k == "m_ev":
                m = list(v) + [0.0] * (4 - len(v))
                P.m_ev = (C.c_double * 4)(*m)
            elif hasattr(P, k):
                setattr(P, k, v)
        self._P = P
        self._keep = {}
        T = OrTables()
        for k in ("lnk", "lna", "T_psi", "T_phi", "dTphi_dlna", "cdf_t", "cdf_F"):
            arr = np.ascontiguousarray(tables[k], dtype=np.float64)
            self._keep[k] = arr
            setattr(T, k, _p(arr, C.c_double))
        T.nk = len(self._keep["lnk"])
        T.na = len(self._keep["lna"])
        T.ncdf = len(self._keep["cdf_t"])
        self._T = T
        self.N = int(self.params["n_grid"])

    # -- background and quadrature -------------------------------------------------
    def hubble(self, a):
        return lib().or_hubble(C.byref(self._P), a)

    def dtau(self, l1, l2):
        return lib().or_dtau(C.byref(self._P), l1, l2)

    def eps_integral(self, m, q, l1, l2, kind):
        return lib().or_eps_integral(C.byref(self._P), m, q, l1, l2, kind)

    def tau(self, a):
        return lib().or_tau(C.byref(self._P), a)

    def lna(self, k):
        return lib().or_lna(C.byref(self._P), float(k))

    def temperature_ev(self):
        return lib().or_temperature_ev(C.byref(self._P))

    # -- sampling ------------------------------------------------------------------
    def sample(self, gidx):
        g = np.ascontiguousarray(gidx, dtype=np.int64)
        n = len(g)
        X = np.zeros(3 * n, np.uint32)
        qs = np.zeros(3 * n, np.float64)
        pm = np.zeros(n, np.float64)
        rc = lib().or_sample(C.byref(self._P), C.byref(self._T), _p(g, C.c_int64), n, _p(X, C.c_uint32),
                             _p(qs, C.c_double), _p(pm, C.c_double))
        if rc != 0:
            raise RuntimeError("oracle sampling failed")
        return X.reshape(3, n), qs.reshape(3, n), pm

    def fd_inverse(self, u):
        return lib().or_fd_inverse(C.byref(self._T), float(u))

    # -- fields ----------------------------------------------------------------------
    def noise(self):
        N = self.N
        R = np.zeros(2 * N ** 3, np.float64)
        lib().or_noise(C.byref(self._P), _p(R, C.c_double))
        return (R[0::2] + 1j * R[1::2]).reshape(N, N, N)

    def fields(self, lna, mask=0xFF, R=None):
        """Real-space fields [8][N][N][N] (z, y, x) at ln a, and max |Im|."""
        N = self.N
        if R is None:
            R = self.noise()
        Rf = np.empty(2 * N ** 3, np.float64)
        Rf[0::2] = R.real.ravel()
        Rf[1::2] = R.imag.ravel()
        out = np.zeros(8 * N ** 3, np.float64)
        mi = C.c_double(0.0)
        lib().or_fields(C.byref(self._P), C.byref(self._T), _p(Rf, C.c_double), lna, mask, _p(out, C.c_double),
                        C.byref(mi))
        return out.reshape(8, N, N, N), mi.value

    def interp_table(self, which, lnk, lna):
        return lib().or_interp_table(C.byref(self._T), _p(self._keep[which], C.c_double), lnk, lna)

    def supersteps(self):
        """The super-step schedule (Sec. 2.1): 1 where the fields are computed."""
        out = np.zeros(self.params["n_steps"] + 1, np.int32)
        lib().or_supersteps(C.byref(self._P), C.byref(self._T), _p(out, C.c_int32))
        return out

    def tf_change(self, j0, j1):
        return lib().or_tf_change(C.byref(self._P), C.byref(self._T), int(j0), int(j1))

    def gather(self, F, x):
        """Read of fields F [8][N][N][N] at one position x (3,), order r = interp_order."""
        Fa = np.ascontiguousarray(F, dtype=np.float64).ravel()
        xa = np.ascontiguousarray(x, dtype=np.float64)
        out = np.zeros(8)
        lib().or_gather(C.byref(self._P), _p(Fa, C.c_double), _p(xa, C.c_double), _p(out, C.c_double))
        return out

    # -- particles ---------------------------------------------------------------------
    def initial(self, gidx, frozen=None):
        g = np.ascontiguousarray(gidx, dtype=np.int64)
        n = len(g)
        X = np.zeros(3 * n, np.uint32)
        qs = np.zeros(3 * n)
        pm = np.zeros(n)
        x = np.zeros(3 * n)
        q = np.zeros(3 * n)
        q0 = np.zeros(3 * n)
        fr = None if frozen is None else np.ascontiguousarray(frozen, dtype=np.float64).ravel()
        rc = lib().or_initial(C.byref(self._P), C.byref(self._T), None if fr is None else _p(fr, C.c_double),
                              _p(g, C.c_int64), n, _p(X, C.c_uint32), _p(qs, C.c_double), _p(pm, C.c_double),
                              _p(x, C.c_double), _p(q, C.c_double), _p(q0, C.c_double))
        if rc != 0:
            raise RuntimeError("oracle initial conditions failed")
        return dict(X=X.reshape(3, n), qs=qs.reshape(3, n), p=pm, x=x.reshape(3, n), q=q.reshape(3, n),
                    q0=q0.reshape(3, n))

    def integrate(self, gidx, x, q, q0, k_from, k_to, frozen=None):
        g = np.ascontiguousarray(gidx, dtype=np.int64)
        n = len(g)
        x = np.ascontiguousarray(x, dtype=np.float64).reshape(3 * n).copy()
        q = np.ascontiguousarray(q, dtype=np.float64).reshape(3 * n).copy()
        q0 = np.ascontiguousarray(q0, dtype=np.float64).reshape(3 * n)
        fr = None if frozen is None else np.ascontiguousarray(frozen, dtype=np.float64).ravel()
        rc = lib().or_integrate(C.byref(self._P), C.byref(self._T), None if fr is None else _p(fr, C.c_double),
                                _p(g, C.c_int64), n, int(k_from), int(k_to), _p(x, C.c_double),
                                _p(q, C.c_double), _p(q0, C.c_double))
        if rc != 0:
            raise RuntimeError("oracle integration failed")
        return x.reshape(3, n), q.reshape(3, n)

    def accel_terms(self, gidx, x, q, k, frozen=None):
        """RMS over the particles of the four terms of eq:releq (-eps grad psi,
        -(q^2/eps) grad phi, q (q.grad phi)/eps, q phi_dot) and of their sum, with the
        fields of step k (Fig. 2)."""
        g = np.ascontiguousarray(gidx, dtype=np.int64)
        n = len(g)
        x = np.ascontiguousarray(x, dtype=np.float64).reshape(3 * n)
        q = np.ascontiguousarray(q, dtype=np.float64).reshape(3 * n)
        fr = None if frozen is None else np.ascontiguousarray(frozen, dtype=np.float64).ravel()
        out = np.zeros(5)
        rc = lib().or_accel_terms(C.byref(self._P), C.byref(self._T), None if fr is None else _p(fr, C.c_double),
                                  _p(g, C.c_int64), n, int(k), _p(x, C.c_double), _p(q, C.c_double),
                                  _p(out, C.c_double))
        if rc != 0:
            raise RuntimeError("oracle acceleration terms failed")
        return out

    def weights(self, q, pmag):
        n = len(pmag)
        q = np.ascontiguousarray(q, dtype=np.float64).reshape(3 * n)
        pm = np.ascontiguousarray(pmag, dtype=np.float64)
        w = np.zeros(n)
        lib().or_weights(C.byref(self._P), n, _p(q, C.c_double), _p(pm, C.c_double), _p(w, C.c_double))
        return w

    def deposit(self, gidx, x, q, w, a, quantity=0):
        g = np.ascontiguousarray(gidx, dtype=np.int64)
        n = len(g)
        x = np.ascontiguousarray(x, dtype=np.float64).reshape(3 * n)
        q = np.ascontiguousarray(q, dtype=np.float64).reshape(3 * n)
        w = np.ascontiguousarray(w, dtype=np.float64)
        N = self.N
        grid = np.zeros(N ** 3)
        lib().or_deposit(C.byref(self._P), _p(g, C.c_int64), n, _p(x, C.c_double), _p(q, C.c_double),
                         _p(w, C.c_double), a, quantity, _p(grid, C.c_double))
        return grid.reshape(N, N, N)

    def run(self, gidx, frozen=None, k_to=None):
        """Sample, transform, integrate to step k_to (default: all steps), weigh."""
        ic = self.initial(gidx, frozen)
        k_to = self.params["n_steps"] if k_to is None else k_to
        x, q = self.integrate(gidx, ic["x"], ic["q"], ic["q0"], 0, k_to, frozen)
        w = self.weights(q, ic["p"])
        return dict(ic, x=x, q=q, w=w)


def philox4x32_10(ctr, key):
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, np.uint32)
    lib().or_philox4x32_10(_p(c, C.c_uint32), _p(k, C.c_uint32), _p(out, C.c_uint32))
    return out


def gauss_legendre(n):
    x = np.zeros(n)
    w = np.zeros(n)
    lib().or_gauss_legendre(n, _p(x, C.c_double), _p(w, C.c_double))
    return x, w


def fd_cdf(t):
    return lib().or_fd_cdf(float(t))


def fft3d_inverse(arr):
    N = arr.shape[0]
    d = np.empty(2 * N ** 3)
    d[0::2] = arr.real.ravel()
    d[1::2] = arr.imag.ravel()
    lib().or_fft3d_inverse(N, _p(d, C.c_double))
    return (d[0::2] + 1j * d[1::2]).reshape(N, N, N)


def dft3d_inverse_naive(arr):
    N = arr.shape[0]
    d = np.empty(2 * N ** 3)
    d[0::2] = arr.real.ravel()
    d[1::2] = arr.imag.ravel()
    out = np.zeros(2 * N ** 3)
    lib().or_dft3d_inverse_naive(N, _p(d, C.c_double), _p(out, C.c_double))
    return (out[0::2] + 1j * out[1::2]).reshape(N, N, N)


def num_threads():
    return lib().or_num_threads()
