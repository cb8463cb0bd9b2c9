"""GPU parity of the hand-written adjoint (gradient) and of the Fisher matrix against the oracle's
dual-number derivatives, plus closed forms, central differences of the GPU log L itself, and the
torch.autograd.Function wrapper (Sec. 2.2, Sec. 2.3 of arXiv:2602.12011)."""
import math

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
    return _lib


def _inj(T):
    return np.array([1e6, 2.0, 0.5, 0.3, 25.8, 0.4, 1.3, 1.375, -1.2108, 2.659, 0.8 * T])


def _setup(O, Lb, dets_T, inj, seed=12011):
    ods, gds = [], []
    for det, T in dets_T:
        k0, nb = W.grid(T)
        od = H.oracle_detector(O, det, T, k0, nb, inj, W.MODE_ALL, seed)
        ods.append(od)
        gds.append(H.library_detector(Lb, od))
    return ods, gds


def _check_grad(O, Lb, ods, gds, th, mask, rel=1e-9, flags=0, name="grad"):
    """Every component against the oracle's Dual<11> gradient on the bar of H.grad_tolerance."""
    g = Lb.loglike_grad(gds, th, mask | flags)
    worst = 0.0
    for s in range(th.shape[0]):
        r = O.loglike(ods, th[s], mask)
        scale = H.scale_of(r["dh"], r["hh"], r["dd"])
        ll, gref = O.grad(ods, th[s], mask)
        F = O.fisher(ods, th[s], mask)
        assert abs(g["logl"][s] - ll) <= 1e-10 * scale
        hh = float(np.sum(r["hh"]))
        for i in range(11):
            tol = H.grad_tolerance(gref[i], hh, F[i, i], rel)
            err = abs(g["grad"][s, i] - gref[i])
            worst = max(worst, err / tol if tol > 0 else 0.0)
            assert err <= tol, (s, W.PARAM_NAMES[i], g["grad"][s, i], gref[i], tol)
    H.record_margin("%s:mask%#x:flags%#x" % (name, mask, flags), worst)


def test_grad_parity_lisa_hm(oracle_mod, Lb):
    T = 2.0 ** 17
    inj = _inj(T)
    ods, gds = _setup(oracle_mod, Lb, [(W.LISA, T)], inj)
    th = np.vstack([inj + np.array([2e3, 0.01, 0.01, -0.02, 0.3, 0.02, 0.05, 1e-3, 1e-3, 0.02, 3.0]),
                    W.draw_prior(5, 51, T)])
    th[2, 0] = 1.5e7          # heavy: the taper region lies inside the band
    _check_grad(oracle_mod, Lb, ods, gds, th, W.MODE_ALL)


def test_grad_parity_tianqin_and_network(oracle_mod, Lb):
    Ts = [(W.LISA, 2.0 ** 17), (W.TAIJI, 2.0 ** 16), (W.TIANQIN, 2.0 ** 16)]
    inj = _inj(2.0 ** 16)
    ods, gds = _setup(oracle_mod, Lb, Ts, inj, seed=7)
    th = np.vstack([inj, W.draw_prior(2, 61, 2.0 ** 16)])
    for fl in (0, Lb.PE_PREC_MIXED):
        _check_grad(oracle_mod, Lb, ods[2:], gds[2:], th, W.MODE_ALL, flags=fl)   # TianQin alone (geocentric)
        _check_grad(oracle_mod, Lb, ods, gds, th, W.MODE_ALL, flags=fl)           # network


def test_grad_single_modes_and_tdi15(oracle_mod, Lb):
    """Each mode alone, and (2,2) with (3,2) (one paired unit), on a TDI 1.5 detector; FP64 and
    PE_PREC_MIXED."""
    T = 2.0 ** 16
    inj = _inj(T)
    det15 = dict(W.LISA, tdi_gen=15)
    ods, gds = _setup(oracle_mod, Lb, [(det15, T)], inj, seed=3)
    th = np.vstack([inj, W.draw_prior(2, 71, T)])
    for mask in (0x01, 0x02, 0x04, 0x08, 0x10, 0x09):
        for fl in (0, Lb.PE_PREC_MIXED):
            _check_grad(oracle_mod, Lb, ods, gds, th, mask, flags=fl)


def test_grad_mixed_precision_forward_pass(oracle_mod, Lb):
    """PE_PREC_MIXED on the gradient: each bin's forward mode sum (log L and the cotangents) comes
    from the mixed-precision unit, and the reverse sweeps run with double-word geometry from a
    double-word tape (mode_bwd_tape_mixed). The oracle bars are the FP64 gradient's, on LISA
    (taper region included) and TianQin (geocentric orbit); the result also stays within 1e-11 of
    the scale of the FP64 call's log L and gradient. PE_PREC_FP32 is refused."""
    T = 2.0 ** 17
    inj = _inj(T)
    ods, gds = _setup(oracle_mod, Lb, [(W.LISA, T)], inj)
    th = np.vstack([inj + np.array([2e3, 0.01, 0.01, -0.02, 0.3, 0.02, 0.05, 1e-3, 1e-3, 0.02, 3.0]),
                    W.draw_prior(5, 51, T)])
    th[2, 0] = 1.5e7
    _check_grad(oracle_mod, Lb, ods, gds, th, W.MODE_ALL, flags=Lb.PE_PREC_MIXED)
    g64 = Lb.loglike_grad(gds, th, W.MODE_ALL)
    gmx = Lb.loglike_grad(gds, th, W.MODE_ALL | Lb.PE_PREC_MIXED)
    worst = 0.0
    for s in range(th.shape[0]):
        r = oracle_mod.loglike(ods, th[s], W.MODE_ALL)
        scale = H.scale_of(r["dh"], r["hh"], r["dd"])
        F = oracle_mod.fisher(ods, th[s], W.MODE_ALL)
        assert abs(gmx["logl"][s] - g64["logl"][s]) <= 1e-11 * scale
        for i in range(11):
            tol = H.grad_tolerance(g64["grad"][s, i], float(np.sum(r["hh"])), F[i, i], 1e-11)
            err = abs(gmx["grad"][s, i] - g64["grad"][s, i])
            worst = max(worst, err / tol)
            assert err <= tol, (s, W.PARAM_NAMES[i])
    H.record_margin("grad_mixed_vs_fp64_1e-11", worst)
    Ts = [(W.TIANQIN, 2.0 ** 16)]
    inj16 = _inj(2.0 ** 16)
    ods, gds = _setup(oracle_mod, Lb, Ts, inj16, seed=7)
    _check_grad(oracle_mod, Lb, ods, gds, np.vstack([inj16, W.draw_prior(2, 61, 2.0 ** 16)]), W.MODE_ALL,
                flags=Lb.PE_PREC_MIXED)
    with pytest.raises(Lb.PeError) as e:
        Lb.loglike_grad(gds, inj16[None, :], W.MODE_ALL | Lb.PE_PREC_FP32)
    assert e.value.status == Lb.PE_EINVAL


def test_grad_matches_central_differences_of_gpu_loglike(oracle_mod, Lb):
    T = 2.0 ** 17
    inj = _inj(T)
    _, gds = _setup(oracle_mod, Lb, [(W.LISA, T)], inj)
    th = inj + np.array([1e3, 0.01, 0.02, -0.02, 0.1, 0.01, 0.05, 0.002, 0.002, 0.01, 2.0])
    g = Lb.loglike_grad(gds, th[None, :], W.MODE_ALL)["grad"][0]
    steps = np.array([1.0, 1e-5, 1e-5, 1e-5, 1e-4, 1e-6, 1e-6, 1e-7, 1e-7, 1e-6, 1e-3])
    for i in range(11):
        tp, tm = th.copy(), th.copy()
        tp[i] += steps[i]
        tm[i] -= steps[i]
        ll = Lb.loglike(gds, np.vstack([tp, tm]), W.MODE_ALL)["logl"]
        fd = (ll[0] - ll[1]) / (2 * steps[i])
        assert g[i] == pytest.approx(fd, rel=2e-4, abs=1e-6 * np.abs(g).max()), W.PARAM_NAMES[i]


def test_grad_out_of_domain_and_bitwise_logl(oracle_mod, Lb):
    T = 2.0 ** 16
    inj = _inj(T)
    _, gds = _setup(oracle_mod, Lb, [(W.LISA, T)], inj)
    th = W.draw_prior(6, 81, T)
    th[2, 1] = 0.3
    g = Lb.loglike_grad(gds, th, W.MODE_ALL, status=True)
    assert g["status"][2] == 1 and np.isneginf(g["logl"][2]) and np.all(g["grad"][2] == 0)
    ll = Lb.loglike(gds, th, W.MODE_ALL)["logl"]
    ok = g["status"] == 0
    assert np.all(np.abs(g["logl"][ok] - ll[ok]) <= 1e-12 * np.abs(ll[ok]))


def test_grad_batch_invariance_bitwise(oracle_mod, Lb):
    """A sample's gradient and log L do not depend on the batch around it, bit for bit, in FP64 and
    PE_PREC_MIXED: each 128-bin tile's partials come from one CTA in a fixed order (the tape is
    private to the thread's column), and the per-sample sums run over the sample's own tiles."""
    T = 2.0 ** 16
    inj = _inj(T)
    _, gds = _setup(oracle_mod, Lb, [(W.LISA, T), (W.TIANQIN, T)], inj, seed=5)
    th = np.vstack([inj, W.draw_prior(7, 97, T)])
    for fl in (0, Lb.PE_PREC_MIXED):
        g = Lb.loglike_grad(gds, th, W.MODE_ALL | fl)
        for s in (0, 3, 7):
            g1 = Lb.loglike_grad(gds, th[s:s + 1], W.MODE_ALL | fl)
            assert np.array_equal(g1["grad"][0], g["grad"][s]), (fl, s)
            assert g1["logl"][0] == g["logl"][s], (fl, s)
        gr = Lb.loglike_grad(gds, th[::-1].copy(), W.MODE_ALL | fl)
        assert np.array_equal(gr["grad"][::-1], g["grad"]), fl


def test_fisher_parity(oracle_mod, Lb):
    T = 2.0 ** 17
    inj = _inj(T)
    ods, gds = _setup(oracle_mod, Lb, [(W.LISA, T)], inj)
    th = np.vstack([inj, W.draw_prior(1, 91, T)])
    F = Lb.fisher(gds, th, W.MODE_ALL)
    for s in range(th.shape[0]):
        Fr = oracle_mod.fisher(ods, th[s], W.MODE_ALL)
        d = np.sqrt(np.abs(np.outer(np.diag(Fr), np.diag(Fr))))
        H.record_margin("fisher_1e-10", np.max(np.abs(F[s] - Fr) / (1e-10 * d)))
        assert np.all(np.abs(F[s] - Fr) <= 1e-10 * d + 1e-300), np.max(np.abs(F[s] - Fr) / d)
        np.testing.assert_array_equal(F[s], F[s].T)


def test_fisher_closed_forms_on_gpu(oracle_mod, Lb):
    """F_dLdL = <h|h>/dL^2 and, for (2,2) alone, F_phi_phi = 4 <h|h> (d h/d phi_c = 2 i h)."""
    T = 2.0 ** 18
    inj = _inj(T)
    _, gds = _setup(oracle_mod, Lb, [(W.LISA, T)], inj)
    F = Lb.fisher(gds, inj[None, :], W.MODE_22)[0]
    hh = Lb.loglike(gds, inj[None, :], W.MODE_22, dhhh=True)["dhhh"][0, :, :, 1].sum()
    assert F[4, 4] == pytest.approx(hh / inj[4] ** 2, rel=1e-10)
    assert F[6, 6] == pytest.approx(4 * hh, rel=1e-10)


def test_autograd_function(oracle_mod, Lb):
    import torch
    from paper_2602_12011_gb300 import autograd as AG
    T = 2.0 ** 16
    inj = _inj(T)
    _, gds = _setup(oracle_mod, Lb, [(W.LISA, T)], inj)
    th = torch.tensor(W.draw_prior(4, 5, T), device="cuda", requires_grad=True)
    ll = AG.loglike(th, gds, W.MODE_ALL)
    w = torch.tensor([1.0, -2.0, 0.5, 3.0], dtype=torch.float64, device="cuda")
    (ll * w).sum().backward()
    ref = Lb.loglike_grad(gds, th.detach(), W.MODE_ALL)
    torch.testing.assert_close(th.grad, w[:, None] * ref["grad"], rtol=0, atol=0)
    torch.testing.assert_close(ll.detach(), ref["logl"], rtol=0, atol=0)


def test_grad_full_size_sampled(oracle_mod, Lb):
    """The gradient over the benchmark batch (T = 2^22 s, B = 1024, 5 modes) in one call, FP64 and
    PE_PREC_MIXED; checked against the oracle's dual-number gradient on the three heaviest samples
    (fewest active bins) and the three lightest (every bin of every mode active: the longest
    in-band signals, the largest phases and t_f ranges)."""
    from concurrent.futures import ThreadPoolExecutor
    wl = W.batch_hm(1024)
    det, T, k0, nb = wl["dets"][0]
    od = H.oracle_detector(oracle_mod, det, T, k0, nb, wl["inj"], wl["inj_mask"], wl["noise_seed"])
    gd = H.library_detector(Lb, od)
    th = wl["theta"]
    mask = wl["mode_mask"]
    g = Lb.loglike_grad([gd], th, mask)
    gm = Lb.loglike_grad([gd], th, mask | Lb.PE_PREC_MIXED)   # mixed forward pass
    assert np.all(np.isfinite(g["grad"])) and np.all(np.isfinite(gm["grad"]))
    order = np.argsort(th[:, 0])
    pick = np.r_[order[-3:], order[:3]]

    def ref(s):          # ctypes releases the GIL: the six samples' oracle calls run in parallel
        r = oracle_mod.loglike([od], th[s], mask)
        return r, oracle_mod.grad([od], th[s], mask)[1], oracle_mod.fisher([od], th[s], mask)

    with ThreadPoolExecutor(max_workers=len(pick)) as ex:
        refs = list(ex.map(ref, pick))
    worst = 0.0
    for s, (r, gref, F) in zip(pick, refs):
        hh = float(np.sum(r["hh"]))
        for i in range(11):
            tol = H.grad_tolerance(gref[i], hh, F[i, i])
            for lab, gg in (("fp64", g), ("mixed", gm)):
                err = abs(gg["grad"][s, i] - gref[i])
                worst = max(worst, err / tol)
                assert err <= tol, (s, th[s, 0], W.PARAM_NAMES[i], lab, err, tol)
    H.record_margin("grad_full_size", worst)
