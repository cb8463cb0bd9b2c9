"""The precision study's FP32 path (mode mask | PE_PREC_FP32, the paper's float32 option, Sec. 3.1).

Every step of the unit runs in FP32, including the TaylorF2 phase, t_f and frac(f t_c). The path
must compute the same quantity as FP64 to FP32 accuracy, stay finite and be bitwise
batch-invariant. It is not expected to meet the 1e-10 parity bar, and it does not: on the full
workload its log L deviates from FP64 by up to ~1e-4 of the likelihood's scale, up to ~2e2 in
absolute terms. The mixed path stays below 1e-14 on the same batch.
"""
import numpy as np
import pytest

from paper_2602_12011_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def Lb():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_2602_12011_gb300 import build as B
    from paper_2602_12011_gb300 import _lib
    B.build()
    _lib.lib()
    return _lib


def test_fp32_signal_per_bin_against_fp64(Lb):
    T = 2.0 ** 18
    k0, nb = W.grid(T)
    th = np.array([3e5, 2.0, 0.5, 0.3, 25.8, 0.4, 1.3, 1.375, -1.2108, 2.659, 0.8 * T])
    for det in (W.LISA, W.TIANQIN):
        d = Lb.Detector(det, T, k0, nb)
        h64 = d.signal(th, W.MODE_ALL)
        h32 = d.signal(th, W.MODE_ALL | Lb.PE_PREC_FP32)
        assert np.all(np.isfinite(h32))
        big = np.abs(h64[0]) > 1e-3 * np.abs(h64[0]).max()
        rel = np.abs(h32[0] - h64[0])[big] / np.abs(h64[0])[big]
        assert np.median(rel) < 1e-3
        assert np.median(rel) > 1e-9          # really FP32 arithmetic


def test_fp32_loglike_full_workload(Lb):
    wl = W.batch_hm(1024)
    det, T, k0, nb = wl["dets"][0]
    g = Lb.Detector(det, T, k0, nb)
    g.inject(wl["inj"], wl["inj_mask"], W.normals(nb, wl["noise_seed"]))
    th = wl["theta"]
    r64 = Lb.loglike([g], th, W.MODE_ALL, dhhh=True)
    r32 = Lb.loglike([g], th, W.MODE_ALL | Lb.PE_PREC_FP32)
    assert np.all(np.isfinite(r32["logl"]))
    sc = 0.5 * g.data_norm().sum() + np.abs(r64["dhhh"][:, 0, :, 0].sum(1)) + 0.5 * r64["dhhh"][:, 0, :, 1].sum(1)
    rel = np.abs(r32["logl"] - r64["logl"]) / sc
    assert rel.max() < 1e-3                   # the same quantity, to FP32 accuracy
    assert rel.max() > 1e-10                  # and it misses the FP64 parity bar
    perm = np.random.Generator(np.random.PCG64(3)).permutation(1024)[:100]
    part = Lb.loglike([g], th[perm], W.MODE_ALL | Lb.PE_PREC_FP32)
    assert np.array_equal(part["logl"], r32["logl"][perm])


def test_precision_flags_are_validated(Lb):
    T = 2.0 ** 16
    d = Lb.Detector(W.LISA, T, *W.grid(T))
    d.set_data(np.zeros((3, d.nb), dtype=np.complex128))
    th = W.draw_prior(2, 1, T)
    with pytest.raises(Lb.PeError) as e:
        Lb.loglike([d], th, W.MODE_ALL | Lb.PE_PREC_FP32 | Lb.PE_PREC_MIXED)
    assert e.value.status == Lb.PE_EINVAL
    with pytest.raises(Lb.PeError) as e:
        Lb.loglike_grad([d], th, W.MODE_ALL | Lb.PE_PREC_FP32)
    assert e.value.status == Lb.PE_EINVAL
