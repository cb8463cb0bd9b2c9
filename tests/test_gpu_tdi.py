"""TDI 1.5 against TDI 2.0 on the GPU (the paper's two FD TDI generations, Sec. 2.1).

TDI 2.0 multiplies each channel's signal by (1 - z^4) and its noise PSD by |1 - z^4|^2, so for the
same noise-free data every whitened product agrees between the two generations: log L, <d|h> and
<h|h> per channel, the SNR, the gradient and the Fisher matrix. The comparison runs both
generations through the library on the same source and prior samples, in FP64 and in the mixed
path, and checks each side against the oracle as well.
"""
import numpy as np
import pytest

from paper_2602_12011_gb300 import workloads as W
from tests import _helpers as H

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


@pytest.fixture(scope="module")
def pair(oracle_mod, Lb):
    T = 2.0 ** 18
    k0, nb = W.grid(T)
    inj = np.array([6e5, 2.5, 0.4, -0.2, 20.0, 0.7, 0.9, 2.1, 0.3, 1.1, 0.8 * T])
    out = {}
    for gen in (15, 20):
        det = dict(W.LISA, tdi_gen=gen)
        od = H.oracle_detector(oracle_mod, det, T, k0, nb, inj, W.MODE_ALL, None)
        out[gen] = (od, H.library_detector(Lb, od))
    th = np.vstack([inj, W.draw_prior(15, 404, T)])
    th[1:, 0] = np.geomspace(2e5, 5e6, 15)
    return out, th, inj


def _scale(g):
    dh, hh = g["dhhh"][:, 0, :, 0], g["dhhh"][:, 0, :, 1]
    return np.abs(dh.sum(1)) + 0.5 * hh.sum(1)


@pytest.mark.parametrize("mixed", [False, True], ids=["fp64", "mixed"])
def test_tdi15_tdi20_likelihood_agree(oracle_mod, Lb, pair, mixed):
    out, th, _ = pair
    m = W.MODE_ALL | (Lb.PE_PREC_MIXED if mixed else 0)
    g15 = Lb.loglike([out[15][1]], th, m, dhhh=True)
    g20 = Lb.loglike([out[20][1]], th, m, dhhh=True)
    dd15, dd20 = out[15][1].data_norm(), out[20][1].data_norm()
    np.testing.assert_allclose(dd20, dd15, rtol=1e-11)
    sc = _scale(g15) + 0.5 * dd15.sum()
    assert np.all(np.abs(g20["logl"] - g15["logl"]) <= 1e-11 * sc)
    assert np.all(np.abs(g20["dhhh"] - g15["dhhh"]).max(axis=(1, 2, 3)) <= 1e-11 * sc)
    # SNR of the injection per channel, the comparison the paper's Sec. 3 setting implies
    snr15 = np.sqrt(g15["dhhh"][0, 0, :, 1])
    snr20 = np.sqrt(g20["dhhh"][0, 0, :, 1])
    np.testing.assert_allclose(snr20, snr15, rtol=1e-11)
    assert snr15[0] > 10
    # each generation against the oracle
    for gen, g in ((15, g15), (20, g20)):
        ll, dhhh = oracle_mod.loglike_batch([out[gen][0]], th[:4], W.MODE_ALL)
        H.assert_loglike_parity({"logl": g["logl"][:4], "dhhh": g["dhhh"][:4]}, ll, dhhh,
                                np.array([out[gen][1].data_norm()]),
                                H.floor_terms(oracle_mod, [out[gen][0]], th[:4], W.MODE_ALL),
                                u=H.U_DW if mixed else H.U64, name="tdi%d" % gen)


def test_tdi15_tdi20_gradient_and_fisher_agree(Lb, pair):
    out, th, inj = pair
    a = Lb.loglike_grad([out[15][1]], th[:6], W.MODE_ALL)
    b = Lb.loglike_grad([out[20][1]], th[:6], W.MODE_ALL)
    F15 = Lb.fisher([out[15][1]], inj[None, :], W.MODE_ALL)[0]
    F20 = Lb.fisher([out[20][1]], inj[None, :], W.MODE_ALL)[0]
    d = np.sqrt(np.abs(np.diag(F15)))
    assert np.all(np.abs(F20 - F15) <= 1e-9 * np.outer(d, d))
    # gradient components on the Fisher scale of each parameter
    sc = np.abs(a["grad"]) + np.sqrt(np.abs(a["logl"]).max() + 1.0) * d[None, :]
    assert np.all(np.abs(b["grad"] - a["grad"]) <= 1e-8 * sc)
