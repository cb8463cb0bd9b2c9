"""ctypes binding of the plain FP64 CPU oracle (``oracle/pe_oracle.cpp``).

TEST INFRASTRUCTURE ONLY: the test suite, ``__graft_entry__.smoke()`` and the CPU-baseline
leg of ``bench.py`` are the only callers. The library under ``paper_2602_12011_gb300`` never
imports this module, and this module never imports the library.

Every function mirrors one exported C function of the oracle; arrays are float64 numpy arrays,
complex values are numpy complex128 (interleaved re, im in memory).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pe_oracle.cpp")
_LIB = os.path.join(_HERE, "build", "liboracle_pe.so")


def build(force: bool = False) -> str:
    """Compile the oracle with the host compiler (-O2, no fast-math, OpenMP over samples)."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    tmp = _LIB + ".tmp%d" % os.getpid()
    subprocess.check_call(["g++", "-O2", "-std=c++17", "-fPIC", "-shared", "-fopenmp", "-o", tmp, _SRC])
    os.replace(tmp, _LIB)
    return _LIB


class OrConfig(C.Structure):
    _fields_ = [
        ("orbit", C.c_int), ("tdi_gen", C.c_int), ("psd_shaping", C.c_int), ("pad_", C.c_int),
        ("arm_m", C.c_double), ("alpha0", C.c_double), ("cartwheel0", C.c_double),
        ("geo_period_s", C.c_double), ("geo_lon", C.c_double), ("geo_lat", C.c_double),
        ("oms_m_rtHz", C.c_double), ("acc_ms2_rtHz", C.c_double),
    ]


class OrDetector(C.Structure):
    _fields_ = [("cfg", OrConfig), ("T", C.c_double), ("k0", C.c_int64), ("nb", C.c_int64),
                ("data", C.c_void_p), ("psd", C.c_void_p)]


def config(d: dict) -> OrConfig:
    """Fill the oracle's configuration struct from a detector dictionary."""
    c = OrConfig()
    c.orbit = int(d["orbit"])
    c.tdi_gen = int(d.get("tdi_gen", 20))
    c.psd_shaping = int(d.get("psd_shaping", 1))
    c.arm_m = float(d["arm_m"])
    c.alpha0 = float(d.get("alpha0", 0.0))
    c.cartwheel0 = float(d.get("cartwheel0", 0.0))
    c.geo_period_s = float(d.get("geo_period_s", 0.0))
    c.geo_lon = float(d.get("geo_lon", 0.0))
    c.geo_lat = float(d.get("geo_lat", 0.0))
    c.oms_m_rtHz = float(d["oms_m_rtHz"])
    c.acc_ms2_rtHz = float(d["acc_ms2_rtHz"])
    return c


_lib = None
_P = C.c_void_p


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


def lib():
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(_LIB)
        L.or_sylm.restype = C.c_double
        L.or_sylm.argtypes = [C.c_int, C.c_int, C.c_double]
        L.or_hhat.argtypes = [C.c_double, C.c_int, C.c_int, C.c_double, _P]
        L.or_psd.argtypes = [C.POINTER(OrConfig), _P, C.c_int64, _P]
        L.or_orbit.argtypes = [C.POINTER(OrConfig), C.c_double, _P]
        L.or_mode.argtypes = [_P, C.c_int, C.c_int, _P, C.c_int64, _P, _P, _P]
        L.or_psi_pn.restype = C.c_double
        L.or_psi_pn.argtypes = [_P, C.c_double]
        L.or_taper.restype = C.c_double
        L.or_taper.argtypes = [_P, C.c_double, C.c_int]
        L.or_polarizations.argtypes = [_P, C.c_uint, _P, C.c_int64, _P, _P]
        L.or_sky_basis.argtypes = [_P, _P, _P, _P]
        L.or_link.argtypes = [C.POINTER(OrConfig), _P, C.c_int, C.c_int, _P, C.c_int64, C.c_int, C.c_int,
                              C.c_double, _P]
        L.or_response.argtypes = [C.POINTER(OrConfig), _P, C.c_uint, _P, C.c_int64, _P]
        L.or_op_count.argtypes = [C.POINTER(OrConfig), _P, C.c_uint, _P, C.c_int64, _P, _P, C.c_double, _P]
        L.or_response_ld.argtypes = [C.POINTER(OrConfig), _P, C.c_uint, _P, C.c_int64, _P]
        L.or_response_xyz.argtypes = [C.POINTER(OrConfig), _P, C.c_uint, _P, C.c_int64, _P]
        L.or_make_data.argtypes = [C.POINTER(OrConfig), _P, C.c_uint, C.c_double, C.c_int64, C.c_int64, _P, _P]
        L.or_loglike.argtypes = [C.POINTER(OrDetector), C.c_int, _P, C.c_uint, _P]
        L.or_loglike_batch.argtypes = [C.POINTER(OrDetector), C.c_int, _P, C.c_int, C.c_uint, C.c_int, _P, _P]
        L.or_max_threads.restype = C.c_int
        L.or_grad.argtypes = [C.POINTER(OrDetector), C.c_int, _P, C.c_uint, _P, _P]
        L.or_grad_batch.argtypes = [C.POINTER(OrDetector), C.c_int, _P, C.c_int, C.c_uint, C.c_int, _P, _P]
        L.or_fisher.argtypes = [C.POINTER(OrDetector), C.c_int, _P, C.c_uint, _P]
        L.or_response_jac.argtypes = [C.POINTER(OrConfig), _P, C.c_uint, _P, C.c_int64, _P]
        _lib = L
    return _lib


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def sylm(l: int, m: int, iota: float) -> float:
    """-2Y_lm(iota, phi=0) from the Wigner-d sum."""
    return lib().or_sylm(l, m, iota)


def hhat(q: float, l: int, m: int, x: float) -> complex:
    """The oracle's leading-order mode factor H_lm(x) for mass ratio q (h_lm ~ H_lm e^{-i m psi})."""
    out = np.zeros(2)
    lib().or_hhat(float(q), l, m, float(x), _ptr(out))
    return complex(out[0], out[1])


def psd(det: dict, f) -> np.ndarray:
    f = _f64(f)
    out = np.zeros((3, f.size))
    c = config(det)
    lib().or_psd(C.byref(c), _ptr(f), f.size, _ptr(out))
    return out


def orbit(det: dict, t: float) -> np.ndarray:
    x = np.zeros((3, 3))
    c = config(det)
    lib().or_orbit(C.byref(c), float(t), _ptr(x))
    return x


def mode(theta, l: int, m: int, f):
    """Returns (H~_lm(f) complex, t_f(f), Psi_lm(f))."""
    th, f = _f64(theta), _f64(f)
    h = np.zeros(2 * f.size)
    tf = np.zeros(f.size)
    ps = np.zeros(f.size)
    lib().or_mode(_ptr(th), l, m, _ptr(f), f.size, _ptr(h), _ptr(tf), _ptr(ps))
    return h.view(np.complex128), tf, ps


def psi_pn(theta, v: float) -> float:
    return lib().or_psi_pn(_ptr(_f64(theta)), float(v))


def taper(theta, f: float, m: int) -> float:
    return lib().or_taper(_ptr(_f64(theta)), float(f), int(m))


def polarizations(theta, mode_mask: int, f):
    th, f = _f64(theta), _f64(f)
    hp = np.zeros(2 * f.size)
    hc = np.zeros(2 * f.size)
    lib().or_polarizations(_ptr(th), mode_mask, _ptr(f), f.size, _ptr(hp), _ptr(hc))
    return hp.view(np.complex128), hc.view(np.complex128)


def sky_basis(theta):
    k = np.zeros(3)
    ep = np.zeros((3, 3))
    ec = np.zeros((3, 3))
    lib().or_sky_basis(_ptr(_f64(theta)), _ptr(k), _ptr(ep), _ptr(ec))
    return k, ep, ec


def link(det: dict, theta, l: int, m: int, f, r: int, s: int, t_fixed: float = float("nan")) -> np.ndarray:
    th, f = _f64(theta), _f64(f)
    out = np.zeros(2 * f.size)
    c = config(det)
    lib().or_link(C.byref(c), _ptr(th), l, m, _ptr(f), f.size, r, s, float(t_fixed), _ptr(out))
    return out.view(np.complex128)


def response(det: dict, theta, mode_mask: int, f) -> np.ndarray:
    """A/E/T response, complex array [3][n]."""
    th, f = _f64(theta), _f64(f)
    out = np.zeros(3 * 2 * f.size)
    c = config(det)
    lib().or_response(C.byref(c), _ptr(th), mode_mask, _ptr(f), f.size, _ptr(out))
    return out.view(np.complex128).reshape(3, f.size)


OP_NAMES = ("add", "mul", "div", "sqrt", "sincos", "exp", "log", "cbrt", "pow", "cmp")


def op_count(det: dict, theta, mode_mask: int, f, data=None, psd=None, T: float = 1.0) -> dict:
    """Operations of the oracle's own steps per active (mode, bin) unit, per active bin and per
    sample (see or_op_count), counted with its operation-counting scalar."""
    th, f = _f64(theta), _f64(f)
    out = np.zeros(2 + 3 * len(OP_NAMES))
    c = config(det)
    dp = None if data is None else np.ascontiguousarray(np.asarray(data, dtype=np.complex128).reshape(3, f.size))
    pp = None if psd is None else _f64(psd).reshape(3, f.size)
    lib().or_op_count(C.byref(c), _ptr(th), mode_mask, _ptr(f), f.size, None if dp is None else _ptr(dp),
                      None if pp is None else _ptr(pp), float(T), _ptr(out))
    k = len(OP_NAMES)
    return {"units": out[0], "bins": out[1], "per_unit": dict(zip(OP_NAMES, out[2:2 + k])),
            "per_bin": dict(zip(OP_NAMES, out[2 + k:2 + 2 * k])), "per_sample": dict(zip(OP_NAMES, out[2 + 2 * k:]))}


def response_ld(det: dict, theta, mode_mask: int, f) -> np.ndarray:
    """The A/E/T response evaluated in long double (the same template), rounded to complex128."""
    th, f = _f64(theta), _f64(f)
    out = np.zeros(3 * 2 * f.size)
    c = config(det)
    lib().or_response_ld(C.byref(c), _ptr(th), mode_mask, _ptr(f), f.size, _ptr(out))
    return out.view(np.complex128).reshape(3, f.size)


def response_xyz(det: dict, theta, mode_mask: int, f) -> np.ndarray:
    th, f = _f64(theta), _f64(f)
    out = np.zeros(3 * 2 * f.size)
    c = config(det)
    lib().or_response_xyz(C.byref(c), _ptr(th), mode_mask, _ptr(f), f.size, _ptr(out))
    return out.view(np.complex128).reshape(3, f.size)


def response_jac(det: dict, theta, mode_mask: int, f) -> np.ndarray:
    """d(Re, Im of A/E/T)/d theta: array [n][3][2][11]."""
    th, f = _f64(theta), _f64(f)
    out = np.zeros((f.size, 3, 2, 11))
    c = config(det)
    lib().or_response_jac(C.byref(c), _ptr(th), mode_mask, _ptr(f), f.size, _ptr(out))
    return out


def make_data(det: dict, theta, mode_mask: int, T: float, k0: int, nb: int, normals=None) -> np.ndarray:
    """Injection + noise (Re/Im ~ N(0, S T/4)); normals [3][nb][2] standard normals or None."""
    th = _f64(theta)
    out = np.zeros((3, nb, 2))
    c = config(det)
    nrm = None if normals is None else _f64(normals).reshape(3, nb, 2)
    lib().or_make_data(C.byref(c), _ptr(th), mode_mask, float(T), int(k0), int(nb),
                       None if nrm is None else _ptr(nrm), _ptr(out))
    return out.view(np.complex128).reshape(3, nb)


class Detector:
    """One detector's grid, data and PSD as the oracle sees them (host arrays)."""

    def __init__(self, det: dict, T: float, k0: int, nb: int, data: np.ndarray, psd_aet: np.ndarray):
        self.det, self.T, self.k0, self.nb = det, float(T), int(k0), int(nb)
        self.data = np.ascontiguousarray(np.asarray(data, dtype=np.complex128).reshape(3, nb))
        self.psd = _f64(psd_aet).reshape(3, nb)

    def struct(self) -> OrDetector:
        s = OrDetector()
        s.cfg = config(self.det)
        s.T, s.k0, s.nb = self.T, self.k0, self.nb
        s.data = self.data.ctypes.data
        s.psd = self.psd.ctypes.data
        return s


def _dets(dets):
    arr = (OrDetector * len(dets))()
    for i, d in enumerate(dets):
        arr[i] = d.struct()
    return arr


def loglike(dets, theta, mode_mask: int) -> dict:
    """Joint log-likelihood; returns logL (component and residual forms) and per-detector sums."""
    th = _f64(theta)
    out = np.zeros(2 + 9 * len(dets))
    lib().or_loglike(_dets(dets), len(dets), _ptr(th), mode_mask, _ptr(out))
    per = out[2:].reshape(len(dets), 3, 3)
    return {"logl": out[0], "logl_resid": out[1], "dh": per[:, 0], "hh": per[:, 1], "dd": per[:, 2]}


def loglike_batch(dets, theta, mode_mask: int, nthreads: int = 0):
    th = _f64(theta).reshape(-1, 11)
    B = th.shape[0]
    logl = np.zeros(B)
    dhhh = np.zeros((B, len(dets), 3, 2))
    lib().or_loglike_batch(_dets(dets), len(dets), _ptr(th), B, mode_mask, int(nthreads), _ptr(logl), _ptr(dhhh))
    return logl, dhhh


def max_threads() -> int:
    return lib().or_max_threads()


def grad(dets, theta, mode_mask: int):
    th = _f64(theta)
    g = np.zeros(11)
    ll = np.zeros(1)
    lib().or_grad(_dets(dets), len(dets), _ptr(th), mode_mask, _ptr(ll), _ptr(g))
    return ll[0], g


def grad_batch(dets, theta, mode_mask: int, nthreads: int = 0):
    th = _f64(theta).reshape(-1, 11)
    B = th.shape[0]
    g = np.zeros((B, 11))
    ll = np.zeros(B)
    lib().or_grad_batch(_dets(dets), len(dets), _ptr(th), B, mode_mask, int(nthreads), _ptr(ll), _ptr(g))
    return ll, g


def fisher(dets, theta, mode_mask: int) -> np.ndarray:
    th = _f64(theta)
    F = np.zeros((11, 11))
    lib().or_fisher(_dets(dets), len(dets), _ptr(th), mode_mask, _ptr(F))
    return F
