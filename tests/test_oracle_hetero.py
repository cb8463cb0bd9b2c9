"""Pins of the oracle's heterodyned (relative-binning) likelihood (oracle/hetero.py).

The heterodyned log L must equal the exact one wherever the per-mode ratio h/h0 is exactly linear
in frequency inside every coarse bin. That holds at the reference itself, and for a change of
distance or of phi_c, where each ratio is a constant. Elsewhere it must converge to the exact log L
as the bins shrink, with the second-order error of linear interpolation. The coarse edges must be
monotone, cover the reference's band and be uniform in the phase metric.
"""
import math

import numpy as np
import pytest

from paper_2602_12011_gb300 import workloads as W

T = 2.0 ** 17
TH0 = np.array([1.5e6, 2.0, 0.4, -0.2, 15.0, 0.6, 0.9, 2.0, 0.4, 1.1, 0.8 * T])


@pytest.fixture(scope="module")
def setup(oracle_mod):
    from oracle import hetero as HT
    k0, nb = W.grid(T)
    f = (k0 + np.arange(nb)) / T
    d = oracle_mod.make_data(W.LISA, TH0, W.MODE_ALL, T, k0, nb, W.normals(nb, 77))
    od = oracle_mod.Detector(W.LISA, T, k0, nb, d, oracle_mod.psd(W.LISA, f))
    return HT, od, k0, nb


def _scale(r):
    return 0.5 * np.sum(r["dd"]) + abs(np.sum(r["dh"])) + 0.5 * np.sum(r["hh"])


def test_default_edges(setup):
    HT, od, k0, nb = setup
    e = HT.default_edges(T, k0, nb, TH0, W.MODE_ALL, 64)
    assert e[0] == 0 and np.all(np.diff(e) > 0)
    fend = HT.band_end(TH0, W.MODE_ALL)
    assert (k0 + e[-1]) / T < fend <= (k0 + e[-1] + 1) / T           # last bin below the band end
    assert 55 <= e.size - 1 <= 64 + 11 * 5
    # every mode's taper marks are edges, and no edge lies past its last mark inside that mode's
    # band (except the last edge)
    fisco = 6.0 ** -1.5 / (2 * math.pi * TH0[0] * HT.MSUN_S)
    for m in (2, 1, 3, 4):
        ks = [int(math.ceil(a * m * fisco * T)) - k0 for a in HT.TAPER_MARKS]
        kend = int(math.ceil(m * fisco * T)) - k0 - 1
        assert all(k in e for k in ks)
        assert not np.any((e[:-1] > ks[-1]) & (e[:-1] <= kend))
    # the metric steps are uniform, up to grid snapping and the added taper edges; only where a
    # single grid bin already spans more than a step (the lowest frequencies) can a step be larger
    fe = (k0 + e) / T
    steps = np.diff(HT.phase_metric(fe, fe[0], fe[-1]))
    total = HT.phase_metric(fe[-1], fe[0], fe[-1]) - HT.phase_metric(fe[0], fe[0], fe[-1])
    width = np.diff(e)
    assert np.all(steps[width > 10] < 1.2 * total / 64)
    # near the low end two targets can snap to one grid bin; the bin above then takes both
    assert np.all(steps[width > 2] < 2.5 * total / 64)


def test_exact_at_reference_and_for_constant_ratios(oracle_mod, setup):
    HT, od, k0, nb = setup
    e = HT.default_edges(T, k0, nb, TH0, W.MODE_ALL, 48)
    het = HT.Hetero(od, TH0, W.MODE_ALL, e)
    for th in (TH0, TH0 * np.r_[1, 1, 1, 1, 1.3, 1, 1, 1, 1, 1, 1], TH0 + np.r_[0, 0, 0, 0, 0, 0, 0.7, 0, 0, 0, 0]):
        ex = oracle_mod.loglike([od], th, W.MODE_ALL)
        ht = het.loglike(th)
        sc = _scale(ex)
        assert abs(ht["logl"] - ex["logl"]) < 1e-11 * sc, (ht["logl"], ex["logl"])
        np.testing.assert_allclose(ht["hh"], ex["hh"][0], rtol=1e-11)
        np.testing.assert_allclose(ht["dh"], ex["dh"][0], rtol=1e-9, atol=1e-11 * sc)


def test_converges_with_bin_count(oracle_mod, setup):
    """Linear interpolation of the ratio: the error shrinks as the bins do (about 4x per halving
    for a single intrinsic parameter: M, q, chi; here all parameters at once)."""
    HT, od, k0, nb = setup
    # an offset in every parameter that costs ~30 in log L at SNR ~ 1300 (a few sigma)
    th = TH0 + 0.05 * np.r_[300.0, 0.002, 0.002, -0.002, 0.0, 0.001, 0.0, 1e-4, 1e-4, 1e-3, 5.0]
    ex = oracle_mod.loglike([od], th, W.MODE_ALL)["logl"]
    err = []
    for n in (64, 128, 256):
        het = HT.Hetero(od, TH0, W.MODE_ALL, HT.default_edges(T, k0, nb, TH0, W.MODE_ALL, n))
        err.append(abs(het.loglike(th)["logl"] - ex))
    # measured: 1.7e-2, 1.0e-2, 1.1e-3 against a log L change of -28
    assert err[2] < 5e-3
    assert err[1] < 0.75 * err[0] and err[2] < 0.5 * err[1]


def test_summary_data_equal_brute_force_interpolant(oracle_mod, setup):
    """The summary-data contraction is exact algebra for the piecewise-linear ratio: building
    h = h0 * r_lin on the fine grid (r_lin interpolated linearly between the edge ratios) and
    summing <d|h>, <h|h> bin by bin gives the same numbers to rounding. A dropped A1, B1 or B2 term,
    or a conjugate on the wrong side, fails this."""
    HT, od, k0, nb = setup
    e = HT.default_edges(T, k0, nb, TH0, W.MODE_ALL, 40)
    het = HT.Hetero(od, TH0, W.MODE_ALL, e)
    th = TH0 + np.r_[50.0, 0.01, 0.01, 0.0, 0.2, 0.01, 0.1, 1e-3, -1e-3, 0.01, 30.0]
    r = het.ratios(th)                                                     # [md][c][edge]
    K = int(e[-1]) + 1
    f = (k0 + np.arange(K)) / T
    h0 = np.array([oracle_mod.response(W.LISA, TH0, 1 << bit, f) for bit in het.modes])
    rl = np.zeros_like(h0)
    for b in range(e.size - 1):
        lo, hi = int(e[b]), int(e[b + 1]) + (1 if b == e.size - 2 else 0)
        slope = (r[:, :, b + 1] - r[:, :, b]) / (het.fe[b + 1] - het.fe[b])
        rl[:, :, lo:hi] = r[:, :, b, None] + slope[:, :, None] * (f[lo:hi] - het.fe[b])
    h = np.sum(h0 * rl, axis=0)                                            # [c][k]
    w = 4.0 / (od.psd[:, :K] * T)
    dh = np.real(np.sum(w * np.conj(od.data[:, :K]) * h, axis=1))
    hh = np.sum(w * np.abs(h) ** 2, axis=1)
    ht = het.loglike(th)
    np.testing.assert_allclose(ht["dh"], dh, rtol=1e-10, atol=1e-10 * np.abs(hh).sum())
    np.testing.assert_allclose(ht["hh"], hh, rtol=1e-10)
