"""ctypes binding of libpespace_gb300.so (include/pespace_gb300.h).

Argument marshalling only: every computation runs in the library's CUDA kernels. The functions
carry the ABI's names. Arrays may be numpy arrays (host) or torch tensors (host or CUDA);
a CUDA tensor's data pointer is passed straight to the library, which works on it in place.
Importing this module does not load the library; the first call does, and it raises if the
library has not been built (there is no CPU fallback).
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "lib", "libpespace_gb300.so")

PE_OK, PE_EINVAL, PE_ENOMEM, PE_ECUDA, PE_ETIMEOUT, PE_ESTATE = range(6)
STATUS_NAMES = {0: "PE_OK", 1: "PE_EINVAL", 2: "PE_ENOMEM", 3: "PE_ECUDA", 4: "PE_ETIMEOUT", 5: "PE_ESTATE"}
NPARAM = 11
# precision flags OR-ed into the mode mask of the forward entry points (see the C header)
PE_PREC_MIXED = 0x100
PE_PREC_FP32 = 0x200


class PeError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__("%s: %s" % (STATUS_NAMES.get(status, str(status)), msg))
        self.status = status


class DetectorConfig(C.Structure):
    _fields_ = [
        ("orbit", C.c_int32), ("tdi_gen", C.c_int32), ("psd_shaping", C.c_int32), ("reserved", C.c_int32),
        ("arm_m", C.c_double), ("alpha0_rad", C.c_double), ("cartwheel0_rad", C.c_double),
        ("geo_period_s", C.c_double), ("geo_lon_rad", C.c_double), ("geo_lat_rad", C.c_double),
        ("oms_m_rtHz", C.c_double), ("acc_ms2_rtHz", C.c_double),
    ]


def config_from_dict(d: dict) -> DetectorConfig:
    c = DetectorConfig()
    c.orbit = int(d["orbit"])
    c.tdi_gen = int(d.get("tdi_gen", 20))
    c.psd_shaping = int(d.get("psd_shaping", 1))
    c.arm_m = float(d["arm_m"])
    c.alpha0_rad = float(d.get("alpha0", 0.0))
    c.cartwheel0_rad = float(d.get("cartwheel0", 0.0))
    c.geo_period_s = float(d.get("geo_period_s", 0.0))
    c.geo_lon_rad = float(d.get("geo_lon", 0.0))
    c.geo_lat_rad = float(d.get("geo_lat", 0.0))
    c.oms_m_rtHz = float(d["oms_m_rtHz"])
    c.acc_ms2_rtHz = float(d["acc_ms2_rtHz"])
    return c


_lib = None
_P = C.c_void_p


def lib():
    """Load the shared library (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libpespace_gb300.so is not built (%s); run __graft_entry__.build()" % LIB_PATH)
        _lib = load(LIB_PATH)
    return _lib


def swap_library(cdll):
    """Route every wrapper of this module through another build of the library (the test build,
    libpespace_gb300_test.so, loaded with load()); returns the previous handle to restore."""
    global _lib
    prev = lib()
    _lib = cdll
    return prev


def load(path: str):
    """A ctypes handle of one build of the library with every signature declared."""
    L = C.CDLL(path)
    L.pe_abi_version.restype = C.c_int
    L.pe_last_error.restype = C.c_char_p
    L.pe_create_detector.argtypes = [C.POINTER(DetectorConfig), C.c_double, C.c_int64, C.c_int64, C.POINTER(_P)]
    L.pe_destroy_detector.argtypes = [_P]
    L.pe_psd_model.argtypes = [_P, _P]
    L.pe_set_data_psd.argtypes = [_P, _P, _P, C.c_int]
    L.pe_data_norm.argtypes = [_P, _P]
    L.pe_signal_aet.argtypes = [_P, _P, C.c_uint, _P, _P]
    L.pe_inject.argtypes = [_P, _P, C.c_uint, _P]
    L.pe_loglike_batch.argtypes = [_P, C.c_int, _P, C.c_int, C.c_uint, _P, _P, _P, _P]
    L.pe_loglike_grad_batch.argtypes = [_P, C.c_int, _P, C.c_int, C.c_uint, _P, _P, _P, _P]
    L.pe_fisher.argtypes = [_P, C.c_int, _P, C.c_int, C.c_uint, _P, _P]
    L.pe_loglike_batch_noalloc.argtypes = [_P, C.c_int, _P, C.c_int, C.c_uint, _P, _P, _P, _P]
    L.pe_loglike_batch_noalloc.restype = C.c_int
    L.pe_plan_create.argtypes = [_P, C.c_int, C.c_int, C.c_uint, _P, _P, _P, _P, C.c_int, C.POINTER(_P)]
    L.pe_plan_launch.argtypes = [_P, _P]
    L.pe_plan_info.argtypes = [_P, _P, _P, _P, _P]
    L.pe_plan_destroy.argtypes = [_P]
    L.pe_autotune.argtypes = [_P, C.c_int, _P, C.c_int, C.c_uint, _P, _P, _P, _P]
    L.pe_tune_set.argtypes = [_P, C.c_int, C.c_int, C.c_uint, C.c_int, C.c_int, C.c_int]
    for name in ("pe_plan_create", "pe_plan_launch", "pe_plan_info", "pe_plan_destroy", "pe_autotune",
                 "pe_tune_set"):
        getattr(L, name).restype = C.c_int
    L.pe_surrogate_create.argtypes = [C.c_uint64, C.POINTER(_P)]
    L.pe_surrogate_destroy.argtypes = [_P]
    L.pe_surrogate_train.argtypes = [_P, _P, C.c_int, C.c_int, C.c_int, C.c_double, _P, _P]
    L.pe_surrogate_set_box.argtypes = [_P, C.c_double, C.c_double, C.c_double, C.c_double]
    L.pe_surrogate_set_node_source.argtypes = [_P, C.c_int]
    L.pe_surrogate_set_node_source.restype = C.c_int
    L.pe_surrogate_set_network_qmax.argtypes = [_P, C.c_double]
    L.pe_surrogate_set_network_qmax.restype = C.c_int
    L.pe_surrogate_targets.argtypes = [_P, C.c_int, _P]
    L.pe_surrogate_predict.argtypes = [_P, _P, C.c_int, _P]
    L.pe_surrogate_loglike_batch.argtypes = [_P, _P, C.c_int, _P, C.c_int, C.c_uint, _P, _P, _P]
    L.pe_surrogate_mismatch.argtypes = [_P, _P, _P, C.c_int, C.c_uint, _P, _P]
    L.pe_set_wait_limit.argtypes = [C.c_double]
    L.pe_set_wait_limit.restype = C.c_int
    L.pe_get_wait_limit.argtypes = []
    L.pe_get_wait_limit.restype = C.c_double
    L.pe_surrogate_mlp_debug.argtypes = [_P, _P, C.c_int, _P, _P, _P]
    L.pe_surrogate_mlp_trace.argtypes = [_P, _P, C.c_int, _P, _P, _P, _P]
    L.pe_surrogate_get_weights.argtypes = [_P, _P, _P]
    L.pe_surrogate_save.argtypes = [_P, C.c_char_p]
    L.pe_surrogate_load.argtypes = [_P, C.c_char_p]
    for name in ("pe_surrogate_create", "pe_surrogate_destroy", "pe_surrogate_train", "pe_surrogate_set_box",
                 "pe_surrogate_targets", "pe_surrogate_predict", "pe_surrogate_loglike_batch",
                 "pe_surrogate_mismatch", "pe_surrogate_mlp_debug", "pe_surrogate_mlp_trace", "pe_surrogate_get_weights",
                 "pe_surrogate_save", "pe_surrogate_load"):
        getattr(L, name).restype = C.c_int
    L.pe_fisher_gaussian.argtypes = [_P, C.c_int, _P, C.c_uint, _P, C.c_int, _P, C.c_int, _P, _P]
    L.pe_fisher_gaussian.restype = C.c_int
    L.pe_hetero_default_edges.argtypes = [C.c_double, C.c_int64, C.c_int64, _P, C.c_uint, C.c_int, _P, _P]
    L.pe_hetero_create.argtypes = [_P, _P, C.c_uint, _P, C.c_int, C.POINTER(_P)]
    L.pe_hetero_loglike_batch.argtypes = [_P, C.c_int, _P, C.c_int, _P, _P, _P, _P]
    L.pe_hetero_destroy.argtypes = [_P]
    for name in ("pe_hetero_default_edges", "pe_hetero_create", "pe_hetero_loglike_batch", "pe_hetero_destroy"):
        getattr(L, name).restype = C.c_int
    L.pe_profile_enable.argtypes = [C.c_int]
    L.pe_profile_read.argtypes = [_P, _P]
    L.pe_measure_fp64_peak.argtypes = [C.c_double, _P]
    L.pe_measure_fp32_peak.argtypes = [C.c_double, _P]
    for name in ("pe_profile_enable", "pe_profile_read", "pe_measure_fp64_peak", "pe_measure_fp32_peak", "pe_create_detector", "pe_destroy_detector", "pe_psd_model", "pe_set_data_psd", "pe_data_norm",
                 "pe_signal_aet", "pe_inject", "pe_loglike_batch", "pe_loglike_grad_batch", "pe_fisher"):
        getattr(L, name).restype = C.c_int
    if hasattr(L, "pe_test_fault_arm"):
        L.pe_test_fault_arm.argtypes = [C.c_int, C.c_long]
        L.pe_test_fault_arm.restype = C.c_int
        for name in ("pe_test_fault_count",):
            getattr(L, name).argtypes = [C.c_int]
            getattr(L, name).restype = C.c_long
        for name in ("pe_test_fault_fired", "pe_test_live_allocations"):
            getattr(L, name).argtypes = []
            getattr(L, name).restype = C.c_long
        L.pe_test_checked_take.argtypes = []
        L.pe_test_checked_take.restype = C.c_int
    return L


def _check(st: int):
    if st != PE_OK:
        raise PeError(st, lib().pe_last_error().decode())


def _ptr(a):
    """Raw data pointer of a numpy array or torch tensor (None passes NULL)."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        return a.ctypes.data
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return a.data_ptr()
    raise TypeError("expected a numpy array or torch tensor, got %r" % type(a))


def _stream(stream):
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


# ---- ABI functions (same names) --------------------------------------------------------------
def pe_set_wait_limit(seconds: float):
    _check(lib().pe_set_wait_limit(float(seconds)))


def pe_get_wait_limit() -> float:
    return lib().pe_get_wait_limit()


def pe_abi_version() -> int:
    return lib().pe_abi_version()


def pe_create_detector(cfg: dict, T_obs: float, k0: int, nbins: int) -> int:
    h = _P()
    c = config_from_dict(cfg)
    _check(lib().pe_create_detector(C.byref(c), float(T_obs), int(k0), int(nbins), C.byref(h)))
    return h.value


def pe_destroy_detector(h: int):
    _check(lib().pe_destroy_detector(h))


def pe_psd_model(h: int, out):
    _check(lib().pe_psd_model(h, _ptr(out)))


def pe_set_data_psd(h: int, data, psd=None, ptr_is_device: bool = False):
    _check(lib().pe_set_data_psd(h, _ptr(data), _ptr(psd), int(bool(ptr_is_device))))


def pe_data_norm(h: int, out):
    _check(lib().pe_data_norm(h, _ptr(out)))


def pe_signal_aet(h: int, theta, mode_mask: int, out, stream=None):
    _check(lib().pe_signal_aet(h, _ptr(theta), int(mode_mask), _ptr(out), _stream(stream)))


def pe_inject(h: int, theta, mode_mask: int, normals=None):
    _check(lib().pe_inject(h, _ptr(theta), int(mode_mask), _ptr(normals)))


def _handles(hs):
    arr = (_P * len(hs))(*hs)
    return arr


def pe_loglike_batch(hs, theta, B: int, mode_mask: int, out_logl, out_dhhh=None, out_status=None, stream=None):
    _check(lib().pe_loglike_batch(_handles(hs), len(hs), _ptr(theta), int(B), int(mode_mask), _ptr(out_logl),
                                  _ptr(out_dhhh), _ptr(out_status), _stream(stream)))


def pe_loglike_batch_noalloc(hs, theta, B: int, mode_mask: int, out_logl, out_dhhh=None, out_status=None,
                             stream=None):
    """pe_loglike_batch with the library's fixed device scratch array: allocates nothing.
    theta and outputs must be CUDA tensors."""
    _check(lib().pe_loglike_batch_noalloc(_handles(hs), len(hs), _ptr(theta), int(B), int(mode_mask),
                                          _ptr(out_logl), _ptr(out_dhhh), _ptr(out_status), _stream(stream)))


def pe_loglike_grad_batch(hs, theta, B: int, mode_mask: int, out_logl, out_grad, out_status=None, stream=None):
    _check(lib().pe_loglike_grad_batch(_handles(hs), len(hs), _ptr(theta), int(B), int(mode_mask), _ptr(out_logl),
                                       _ptr(out_grad), _ptr(out_status), _stream(stream)))


def pe_fisher(hs, theta, B: int, mode_mask: int, out_F, stream=None):
    _check(lib().pe_fisher(_handles(hs), len(hs), _ptr(theta), int(B), int(mode_mask), _ptr(out_F),
                           _stream(stream)))


def pe_profile_enable(on: bool):
    _check(lib().pe_profile_enable(int(bool(on))))


def pe_profile_read():
    """(summed device ms, launches) of the fused kernels since the previous read."""
    ms = C.c_double()
    n = C.c_int64()
    _check(lib().pe_profile_read(C.addressof(ms), C.addressof(n)))
    return ms.value, n.value


def pe_measure_fp64_peak(seconds: float = 1.0) -> float:
    t = C.c_double()
    _check(lib().pe_measure_fp64_peak(float(seconds), C.addressof(t)))
    return t.value


def pe_measure_fp32_peak(seconds: float = 1.0) -> float:
    t = C.c_double()
    _check(lib().pe_measure_fp32_peak(float(seconds), C.addressof(t)))
    return t.value


# ---- convenience object ------------------------------------------------------------------------
class Detector:
    """One detector handle with its grid f_k = k/T, k in [k0, k0 + nbins)."""

    def __init__(self, cfg: dict, T_obs: float, k0: int, nbins: int):
        self.cfg, self.T, self.k0, self.nb = dict(cfg), float(T_obs), int(k0), int(nbins)
        self.handle = pe_create_detector(cfg, T_obs, k0, nbins)

    def close(self):
        if self.handle:
            pe_destroy_detector(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def psd(self) -> np.ndarray:
        out = np.zeros((3, self.nb))
        pe_psd_model(self.handle, out)
        return out

    def set_data(self, data, psd=None):
        """data: complex [3][nb] (numpy) or a device tensor of float64 [3][nb][2]."""
        if isinstance(data, np.ndarray):
            d = np.ascontiguousarray(data.astype(np.complex128).reshape(3, self.nb))
            p = None if psd is None else np.ascontiguousarray(np.asarray(psd, dtype=np.float64).reshape(3, self.nb))
            pe_set_data_psd(self.handle, d, p, False)
        else:
            pe_set_data_psd(self.handle, data, psd, True)

    def inject(self, theta, mode_mask: int, normals=None):
        th = np.ascontiguousarray(np.asarray(theta, dtype=np.float64))
        n = None if normals is None else np.ascontiguousarray(np.asarray(normals, dtype=np.float64))
        pe_inject(self.handle, th, mode_mask, n)

    def data_norm(self) -> np.ndarray:
        out = np.zeros(3)
        pe_data_norm(self.handle, out)
        return out

    def signal(self, theta, mode_mask: int) -> np.ndarray:
        th = np.ascontiguousarray(np.asarray(theta, dtype=np.float64))
        out = np.zeros((3, self.nb), dtype=np.complex128)
        pe_signal_aet(self.handle, th, mode_mask, out)
        return out


def loglike(dets, theta, mode_mask: int, dhhh: bool = False, status: bool = False, stream=None):
    """Batched joint log-likelihood. theta: numpy [B][11] (host path) or CUDA tensor [B][11]
    (device path, outputs are CUDA tensors on the same stream)."""
    hs = [d.handle for d in dets]
    if isinstance(theta, np.ndarray):
        th = np.ascontiguousarray(theta.reshape(-1, NPARAM).astype(np.float64))
        B = th.shape[0]
        out = np.zeros(B)
        dh = np.zeros((B, len(dets), 3, 2)) if dhhh else None
        stt = np.zeros(B, dtype=np.int32) if status else None
        pe_loglike_batch(hs, th, B, mode_mask, out, dh, stt, stream)
    else:
        import torch
        th = theta.reshape(-1, NPARAM).contiguous()
        B = th.shape[0]
        out = torch.empty(B, dtype=torch.float64, device=th.device)
        dh = torch.empty((B, len(dets), 3, 2), dtype=torch.float64, device=th.device) if dhhh else None
        stt = torch.empty(B, dtype=torch.int32, device=th.device) if status else None
        if stream is None:
            stream = torch.cuda.current_stream(th.device)
        pe_loglike_batch(hs, th, B, mode_mask, out, dh, stt, stream)
    res = {"logl": out}
    if dhhh:
        res["dhhh"] = dh
    if status:
        res["status"] = stt
    return res


def loglike_grad(dets, theta, mode_mask: int, status: bool = False, stream=None):
    """Batched log-likelihood and its gradient d logL/d theta [B][11] (hand-written adjoint).
    theta: numpy [B][11] (host path) or CUDA tensor (device path, outputs on the same stream)."""
    hs = [d.handle for d in dets]
    if isinstance(theta, np.ndarray):
        th = np.ascontiguousarray(theta.reshape(-1, NPARAM).astype(np.float64))
        B = th.shape[0]
        ll = np.zeros(B)
        g = np.zeros((B, NPARAM))
        stt = np.zeros(B, dtype=np.int32) if status else None
    else:
        import torch
        th = theta.reshape(-1, NPARAM).contiguous()
        B = th.shape[0]
        ll = torch.empty(B, dtype=torch.float64, device=th.device)
        g = torch.empty((B, NPARAM), dtype=torch.float64, device=th.device)
        stt = torch.empty(B, dtype=torch.int32, device=th.device) if status else None
        if stream is None:
            stream = torch.cuda.current_stream(th.device)
    pe_loglike_grad_batch(hs, th, B, mode_mask, ll, g, stt, stream)
    res = {"logl": ll, "grad": g}
    if status:
        res["status"] = stt
    return res


def fisher(dets, theta, mode_mask: int, stream=None):
    """Fisher matrices F[B][11][11] = <dh/dtheta_i | dh/dtheta_j> (summed over detectors, channels)."""
    hs = [d.handle for d in dets]
    if isinstance(theta, np.ndarray):
        th = np.ascontiguousarray(theta.reshape(-1, NPARAM).astype(np.float64))
        B = th.shape[0]
        F = np.zeros((B, NPARAM, NPARAM))
    else:
        import torch
        th = theta.reshape(-1, NPARAM).contiguous()
        B = th.shape[0]
        F = torch.empty((B, NPARAM, NPARAM), dtype=torch.float64, device=th.device)
        if stream is None:
            stream = torch.cuda.current_stream(th.device)
    pe_fisher(hs, th, B, mode_mask, F, stream)
    return F


def pe_plan_create(hs, theta, B: int, mode_mask: int, out_logl, out_dhhh=None, out_status=None,
                   autotune: bool = True) -> int:
    h = _P()
    _check(lib().pe_plan_create(_handles(hs), len(hs), int(B), int(mode_mask), _ptr(theta), _ptr(out_logl),
                                _ptr(out_dhhh), _ptr(out_status), int(bool(autotune)), C.byref(h)))
    return h.value


def pe_plan_launch(plan: int, stream=None):
    _check(lib().pe_plan_launch(plan, _stream(stream)))


def pe_plan_info(plan: int):
    v, c, r, ms = C.c_int(), C.c_int(), C.c_int(), C.c_double()
    _check(lib().pe_plan_info(plan, C.addressof(v), C.addressof(c), C.addressof(r), C.addressof(ms)))
    return {"fwd_variant": v.value, "ctas_per_sm": c.value, "subtiles": r.value, "tuned_ms": ms.value}


def pe_plan_destroy(plan: int):
    _check(lib().pe_plan_destroy(plan))


def pe_autotune(hs, theta, B: int, mode_mask: int):
    v, c, r, ms = C.c_int(), C.c_int(), C.c_int(), C.c_double()
    _check(lib().pe_autotune(_handles(hs), len(hs), _ptr(theta), int(B), int(mode_mask), C.addressof(v),
                             C.addressof(c), C.addressof(r), C.addressof(ms)))
    return {"fwd_variant": v.value, "ctas_per_sm": c.value, "subtiles": r.value, "tuned_ms": ms.value}


def pe_tune_set(hs, B: int, mode_mask: int, fwd_variant: int, ctas_per_sm: int, subtiles: int):
    _check(lib().pe_tune_set(_handles(hs), len(hs), int(B), int(mode_mask), int(fwd_variant), int(ctas_per_sm),
                             int(subtiles)))


class Plan:
    """A CUDA-graph plan of the batched log-likelihood over fixed device buffers: refill
    ``theta`` in place, then ``launch()``; ``logl`` (and ``dhhh``) hold the results."""

    def __init__(self, dets, B: int, mode_mask: int, theta=None, dhhh: bool = False, autotune: bool = True):
        import torch
        self.dets = list(dets)
        self.B = int(B)
        self.theta = theta if theta is not None else torch.zeros((B, NPARAM), dtype=torch.float64, device="cuda")
        self.logl = torch.empty(B, dtype=torch.float64, device=self.theta.device)
        self.dhhh = torch.empty((B, len(dets), 3, 2), dtype=torch.float64, device=self.theta.device) if dhhh else None
        self.status = torch.empty(B, dtype=torch.int32, device=self.theta.device)
        self.handle = pe_plan_create([d.handle for d in self.dets], self.theta, B, mode_mask, self.logl, self.dhhh,
                                     self.status, autotune)

    def launch(self, stream=None):
        import torch
        pe_plan_launch(self.handle, stream if stream is not None else torch.cuda.current_stream(self.theta.device))

    def info(self):
        return pe_plan_info(self.handle)

    def close(self):
        if getattr(self, "handle", None):
            pe_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---- learned surrogate ---------------------------------------------------------------------------
SUR_NODES = 256
SUR_NOUT = 5 * 2 * SUR_NODES
SUR_NIN = 64


class Surrogate:
    """The BF16 tensor-core MLP surrogate with its node-spline likelihood path (device tensors)."""

    def __init__(self, seed: int = 2605):
        h = _P()
        _check(lib().pe_surrogate_create(int(seed), C.byref(h)))
        self.handle = h.value

    def close(self):
        if getattr(self, "handle", None):
            _check(lib().pe_surrogate_destroy(self.handle))
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_box(self, mtot_lo: float, mtot_hi: float, q_max: float = 10.0, chi_max: float = 0.99):
        _check(lib().pe_surrogate_set_box(self.handle, float(mtot_lo), float(mtot_hi), float(q_max), float(chi_max)))

    def set_network_qmax(self, q_net: float):
        """Largest mass ratio whose node values come from the network (exact node values above)."""
        _check(lib().pe_surrogate_set_network_qmax(self.handle, float(q_net)))

    def set_node_source(self, source: int):
        """0: network node values (default); 1: plain generator's node values (no network)."""
        _check(lib().pe_surrogate_set_node_source(self.handle, int(source)))

    def train(self, theta, epochs: int, batch: int = 1024, lr: float = 1e-3):
        """theta: CUDA float64 tensor [n][11]. Returns (final loss, per-epoch loss curve)."""
        n = int(theta.shape[0])
        loss = C.c_double()
        curve = np.zeros(epochs, dtype=np.float32)
        _check(lib().pe_surrogate_train(self.handle, _ptr(theta.contiguous()), n, int(epochs), int(batch), float(lr),
                                        C.addressof(loss), curve.ctypes.data))
        return loss.value, curve

    def predict(self, theta):
        import torch
        out = torch.empty((theta.shape[0], SUR_NOUT), dtype=torch.float32, device=theta.device)
        _check(lib().pe_surrogate_predict(self.handle, _ptr(theta.contiguous()), int(theta.shape[0]), _ptr(out)))
        return out

    @staticmethod
    def targets(theta):
        import torch
        out = torch.empty((theta.shape[0], SUR_NOUT), dtype=torch.float32, device=theta.device)
        _check(lib().pe_surrogate_targets(_ptr(theta.contiguous()), int(theta.shape[0]), _ptr(out)))
        return out

    def loglike(self, dets, theta, mode_mask: int, stream=None):
        import torch
        B = int(theta.shape[0])
        out = torch.empty(B, dtype=torch.float64, device=theta.device)
        used = torch.empty(B, dtype=torch.int32, device=theta.device)
        st = stream if stream is not None else torch.cuda.current_stream(theta.device)
        _check(lib().pe_surrogate_loglike_batch(self.handle, _handles([d.handle for d in dets]), len(dets),
                                                _ptr(theta.contiguous()), B, int(mode_mask), _ptr(out), _ptr(used),
                                                _stream(st)))
        return out, used

    def mismatch(self, det, theta, mode_mask: int, stream=None):
        import torch
        B = int(theta.shape[0])
        out = torch.empty(B, dtype=torch.float64, device=theta.device)
        st = stream if stream is not None else torch.cuda.current_stream(theta.device)
        _check(lib().pe_surrogate_mismatch(self.handle, det.handle, _ptr(theta.contiguous()), B, int(mode_mask),
                                           _ptr(out), _stream(st)))
        return out

    def weights(self) -> np.ndarray:
        n = C.c_int64()
        _check(lib().pe_surrogate_get_weights(self.handle, None, C.addressof(n)))
        w = np.zeros(n.value, dtype=np.float32)
        _check(lib().pe_surrogate_get_weights(self.handle, w.ctypes.data, C.addressof(n)))
        return w

    def mlp_debug(self, x: np.ndarray, dy: np.ndarray):
        """Forward + backward on host inputs x [B][64] and cotangents dy [B][2560] (fp32)."""
        x = np.ascontiguousarray(x, dtype=np.float32)
        dy = np.ascontiguousarray(dy, dtype=np.float32)
        B = x.shape[0]
        y = np.zeros((B, SUR_NOUT), dtype=np.float32)
        g = np.zeros_like(self.weights())
        _check(lib().pe_surrogate_mlp_debug(self.handle, x.ctypes.data, B, dy.ctypes.data, y.ctypes.data, g.ctypes.data))
        return y, g

    # sizes of the intermediates pe_surrogate_mlp_trace returns, per row, in order
    TRACE_LAYOUT = (("X", 64), ("Z0", 256), ("H0", 256), ("Z1", 256), ("H1", 256), ("Z2", 256), ("H2", 256),
                    ("Y", 2560), ("dH2", 256), ("dZ2", 256), ("dZb2", 256), ("dH1", 256), ("dZ1", 256),
                    ("dZb1", 256), ("dH0", 256), ("dZ0", 256), ("dZb0", 256))

    def mlp_trace(self, x: np.ndarray, dy: np.ndarray):
        """mlp_debug plus every intermediate of the pass: returns y, grads and a dict name -> [B][n]."""
        x = np.ascontiguousarray(x, dtype=np.float32)
        dy = np.ascontiguousarray(dy, dtype=np.float32)
        B = x.shape[0]
        y = np.zeros((B, SUR_NOUT), dtype=np.float32)
        g = np.zeros_like(self.weights())
        tr = np.zeros(B * sum(n for _, n in self.TRACE_LAYOUT), dtype=np.float32)
        _check(lib().pe_surrogate_mlp_trace(self.handle, x.ctypes.data, B, dy.ctypes.data, y.ctypes.data,
                                            g.ctypes.data, tr.ctypes.data))
        out, o = {}, 0
        for name, n in self.TRACE_LAYOUT:
            out[name] = tr[o:o + B * n].reshape(B, n)
            o += B * n
        return y, g, out

    def save(self, path: str):
        _check(lib().pe_surrogate_save(self.handle, path.encode()))

    def load(self, path: str):
        _check(lib().pe_surrogate_load(self.handle, path.encode()))


def fisher_gaussian(dets, theta0, mode_mask: int, idx, normals=None):
    """Fisher-Gaussian posterior on the parameters idx (others fixed at theta0): returns
    (cov [k][k], samples [n][11]) with samples = theta0 + L z for the given standard normals z [n][k]."""
    th = np.ascontiguousarray(np.asarray(theta0, dtype=np.float64).reshape(NPARAM))
    ix = np.ascontiguousarray(np.asarray(idx, dtype=np.int32))
    k = ix.size
    cov = np.zeros((k, k))
    if normals is None:
        n, z, out = 0, None, None
    else:
        z = np.ascontiguousarray(np.asarray(normals, dtype=np.float64).reshape(-1, k))
        n = z.shape[0]
        out = np.zeros((n, NPARAM))
    _check(lib().pe_fisher_gaussian(_handles([d.handle for d in dets]), len(dets), _ptr(th), int(mode_mask), _ptr(ix),
                                    k, _ptr(z), n, _ptr(cov), _ptr(out)))
    return cov, out


# ---- heterodyned (relative-binning) likelihood ------------------------------------------------------
def pe_hetero_default_edges(T_obs: float, k0: int, nbins: int, theta0, mode_mask: int, nbins_coarse: int) -> np.ndarray:
    """Coarse-bin edges (fine-bin indices) for reference theta0; host computation, no GPU needed."""
    th = np.ascontiguousarray(np.asarray(theta0, dtype=np.float64))
    cap = nbins_coarse + 64
    out = np.zeros(cap, dtype=np.int64)
    n = C.c_int(cap)
    _check(lib().pe_hetero_default_edges(float(T_obs), int(k0), int(nbins), _ptr(th), int(mode_mask),
                                         int(nbins_coarse), _ptr(out), C.byref(n)))
    return out[:n.value].copy()


class Hetero:
    """Summary data of one detector (with data set) for a reference theta0 and coarse edges (fine-bin
    indices; default: pe_hetero_default_edges with nbins_coarse bins). The detector must stay open."""

    def __init__(self, det, theta0, mode_mask: int, edges=None, nbins_coarse: int = 256):
        th = np.ascontiguousarray(np.asarray(theta0, dtype=np.float64))
        if edges is None:
            edges = pe_hetero_default_edges(det.T, det.k0, det.nb, th, mode_mask, nbins_coarse)
        self.edges = np.ascontiguousarray(np.asarray(edges, dtype=np.int64))
        self.det = det
        h = _P()
        _check(lib().pe_hetero_create(det.handle, _ptr(th), int(mode_mask), _ptr(self.edges), int(self.edges.size),
                                      C.byref(h)))
        self.handle = h.value

    def close(self):
        if getattr(self, "handle", None):
            lib().pe_hetero_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def pe_hetero_loglike_batch(hs, theta, B: int, out_logl, out_dhhh=None, out_status=None, stream=None):
    _check(lib().pe_hetero_loglike_batch(_handles(hs), len(hs), _ptr(theta), int(B), _ptr(out_logl), _ptr(out_dhhh),
                                         _ptr(out_status), _stream(stream)))


def hetero_loglike(hets, theta, dhhh: bool = False, status: bool = False, stream=None):
    """Heterodyned log L of a batch (numpy host path or CUDA tensors, as loglike)."""
    hs = [h.handle for h in hets]
    if isinstance(theta, np.ndarray):
        th = np.ascontiguousarray(theta.reshape(-1, NPARAM).astype(np.float64))
        B = th.shape[0]
        ll = np.zeros(B)
        dh = np.zeros((B, len(hs), 3, 2)) if dhhh else None
        st = np.zeros(B, dtype=np.int32) if status else None
    else:
        import torch
        th = theta.reshape(-1, NPARAM).contiguous()
        B = th.shape[0]
        ll = torch.empty(B, dtype=torch.float64, device=th.device)
        dh = torch.empty((B, len(hs), 3, 2), dtype=torch.float64, device=th.device) if dhhh else None
        st = torch.empty(B, dtype=torch.int32, device=th.device) if status else None
        if stream is None:
            stream = torch.cuda.current_stream(th.device)
    pe_hetero_loglike_batch(hs, th, B, ll, dh, st, stream)
    res = {"logl": ll}
    if dhhh:
        res["dhhh"] = dh
    if status:
        res["status"] = st
    return res
