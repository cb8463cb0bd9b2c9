"""GPU parity of the mixed FP64/double-word forward path (mode mask | PE_PREC_MIXED).

The TaylorF2 phase, t_f, the angle reductions and the sums stay FP64; the response geometry runs
in double-word FP32 arithmetic. The mixed path is held to the same oracle bars as the FP64 path
(per-bin signal; log L and its <d|h>, <h|h> parts to 1e-10 of the likelihood's scale, Eq.
eq_ll_fd), on the same seeded inputs: ragged small grids, edge grids, the three-detector network,
and sampled outputs of the full T = 2^22 s, B = 1024 workload in one batched launch. It is also
compared with the GPU's own FP64 path per bin, checked for bitwise batch invariance, and run
through a plan (the no-allocation entry point is checked in its own file, collected last).
"""
import numpy as np
import pytest

from paper_2602_12011_gb300 import workloads as W
from tests import _helpers as H

pytestmark = pytest.mark.gpu

MIX = 0x100


@pytest.fixture(scope="module")
def Lb():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_2602_12011_gb300 import build as B
    from paper_2602_12011_gb300 import _lib
    B.build()
    _lib.lib()
    assert _lib.PE_PREC_MIXED == MIX
    return _lib


def _th_small(T):
    return np.array([1e6, 2.0, 0.5, 0.3, 25.8, 0.4, 1.3, 1.375, -1.2108, 2.659, 0.8 * T])


def _od_dd(O, od):
    return O.loglike([od], np.array([1e6, 2, 0, 0, 1, 0, 0, 0, 0, 0, 0.0]), 0)["dd"]


@pytest.mark.parametrize("det", [W.LISA, W.TAIJI, W.TIANQIN, dict(W.LISA, tdi_gen=15)],
                         ids=["lisa", "taiji", "tianqin", "lisa15"])
@pytest.mark.parametrize("mask", [W.MODE_22, W.MODE_ALL, 0x02, 0x10])
def test_mixed_signal_per_bin(oracle_mod, Lb, det, mask):
    """Every bin of the mixed A/E/T signal against the oracle (the FP64 path's per-bin bar), and
    against the GPU FP64 path to the double-word rounding level."""
    T = 2.0 ** 18
    k0, nb = W.grid(T)
    th = _th_small(T)
    th[0] = 3e5
    d = Lb.Detector(det, T, k0, nb)
    hm = d.signal(th, mask | MIX)
    h64 = d.signal(th, mask)
    ref = oracle_mod.response(det, th, mask, H.grid_f(T, k0, nb))
    phi = H.phase_magnitude(oracle_mod, th, mask, H.grid_f(T, k0, nb))
    H.assert_signal_parity(hm, ref, "mixed_signal_per_bin:%s:%s:%#x" % (det["name"], det["tdi_gen"], mask), phi,
                           u=H.U_DW)
    for c in range(3):
        # double words carry ~48-bit significands: a chain of ~100 operations stays near 1e-13 of
        # the single-link terms. At long wavelength (a = pi f L << 1) the TDI channels are O(a^2)
        # times those terms, so rounding in either path shows up amplified by 1/a^2 there.
        e64 = np.abs(hm[c] - h64[c])
        ae64 = np.maximum(np.abs(h64[0]), np.abs(h64[1]))
        a2 = (np.pi * H.grid_f(T, k0, nb) * det["arm_m"] / 299792458.0) ** 2
        tol64 = 1e-11 * np.abs(h64[c]) + 1e-12 * ae64 + 2e-14 * ae64 / a2 + 1e-14 * np.abs(h64[c]).max()
        assert np.all(e64 <= tol64), (c, np.max(e64 / (np.abs(h64[c]) + 1e-300)))


@pytest.mark.parametrize("T,nbad", [(2.0 ** 14, 0), (2.0 ** 17, 3)])
def test_mixed_loglike_small_grids(oracle_mod, Lb, T, nbad):
    k0, nb = W.grid(T)
    od = H.oracle_detector(oracle_mod, W.LISA, T, k0, nb, _th_small(T), W.MODE_ALL, 11)
    gd = H.library_detector(Lb, od)
    th = W.draw_prior(24, 77, T)
    th[:, 0] = np.geomspace(1e5, 1e7, 24)
    for i in range(nbad):
        th[3 * i + 1, [1, 2, 4][i]] = [0.5, 1.2, -1.0][i]
    g = Lb.loglike([gd], th, W.MODE_ALL | MIX, dhhh=True, status=True)
    ll, dhhh = oracle_mod.loglike_batch([od], th, W.MODE_ALL)
    bad = g["status"] != 0
    assert bad.sum() == nbad
    assert np.all(np.isneginf(g["logl"][bad]))
    good = ~bad
    H.assert_loglike_parity({"logl": g["logl"][good], "dhhh": g["dhhh"][good]}, ll[good], dhhh[good],
                            _od_dd(oracle_mod, od), H.floor_terms(oracle_mod, [od], th[good], W.MODE_ALL), u=H.U_DW,
                            name="mixed")


def test_mixed_loglike_edge_grids(oracle_mod, Lb):
    T = 2.0 ** 16
    for k0, nb in ((700, 1), (100, 128), (3000, 37)):
        od = H.oracle_detector(oracle_mod, W.LISA, T, k0, nb, _th_small(T), W.MODE_ALL, 3)
        gd = H.library_detector(Lb, od)
        th = np.vstack([_th_small(T), _th_small(T)])
        th[1, 0] = 1e5
        g = Lb.loglike([gd], th, W.MODE_ALL | MIX, dhhh=True)
        ll, dhhh = oracle_mod.loglike_batch([od], th, W.MODE_ALL)
        H.assert_loglike_parity(g, ll, dhhh, _od_dd(oracle_mod, od), H.floor_terms(oracle_mod, [od], th, W.MODE_ALL),
                                u=H.U_DW, name="mixed")


def test_mixed_single_source_full_grid(oracle_mod, Lb):
    wl = W.single_22()
    det, T, k0, nb = wl["dets"][0]
    od = H.oracle_detector(oracle_mod, det, T, k0, nb, wl["inj"], wl["inj_mask"], wl["noise_seed"])
    gd = H.library_detector(Lb, od)
    th = np.vstack([wl["inj"], wl["inj"] + np.array([1e2, 1e-3, 0, 0, 0.1, 0.01, 0.1, 1e-3, 1e-3, 0.01, 5.0])])
    g = Lb.loglike([gd], th, wl["mode_mask"] | MIX, dhhh=True)
    ll, dhhh = oracle_mod.loglike_batch([od], th, wl["mode_mask"])
    H.assert_loglike_parity(g, ll, dhhh, _od_dd(oracle_mod, od), H.floor_terms(oracle_mod, [od], th, wl["mode_mask"]),
                            u=H.U_DW, name="mixed")


def test_mixed_network(oracle_mod, Lb):
    Ts = (2.0 ** 19, 2.0 ** 18, 2.0 ** 17)
    ods, gds = [], []
    inj = _th_small(2.0 ** 17)
    for det, T in zip((W.LISA, W.TAIJI, W.TIANQIN), Ts):
        k0, nb = W.grid(T)
        od = H.oracle_detector(oracle_mod, det, T, k0, nb, inj, W.MODE_ALL, 21)
        ods.append(od)
        gds.append(H.library_detector(Lb, od))
    th = np.vstack([inj, W.draw_prior(6, 99, 2.0 ** 17)])
    g = Lb.loglike(gds, th, W.MODE_ALL | MIX, dhhh=True)
    ll, dhhh = oracle_mod.loglike_batch(ods, th, W.MODE_ALL)
    dd = np.array([_od_dd(oracle_mod, od)[0] for od in ods])
    H.assert_loglike_parity(g, ll, dhhh, dd, H.floor_terms(oracle_mod, ods, th, W.MODE_ALL), u=H.U_DW, name="mixed")


def test_mixed_full_size_sampled(oracle_mod, Lb):
    """LISA, 5 modes, T = 2^22 s (209,296 bins), B = 1024 in one launch; 16 samples checked."""
    wl = W.batch_hm(1024)
    det, T, k0, nb = wl["dets"][0]
    od = H.oracle_detector(oracle_mod, det, T, k0, nb, wl["inj"], wl["inj_mask"], wl["noise_seed"])
    gd = H.library_detector(Lb, od)
    th = wl["theta"]
    g = Lb.loglike([gd], th, wl["mode_mask"] | MIX, dhhh=True)
    assert np.all(np.isfinite(g["logl"]))
    order = np.argsort(th[:, 0])
    pick = np.unique(np.r_[order[:3], order[np.linspace(200, 1023, 13).astype(int)]])
    ll, dhhh = oracle_mod.loglike_batch([od], th[pick], wl["mode_mask"])
    H.assert_loglike_parity({"logl": g["logl"][pick], "dhhh": g["dhhh"][pick]}, ll, dhhh, _od_dd(oracle_mod, od),
                            H.floor_terms(oracle_mod, [od], th[pick], wl["mode_mask"]), u=H.U_DW, name="mixed")
    # every sample against the GPU FP64 path, on the same scale
    g64 = Lb.loglike([gd], th, wl["mode_mask"], dhhh=True)
    sc = 0.5 * gd.data_norm().sum() + np.abs(g64["dhhh"][:, 0, :, 0].sum(1)) + 0.5 * g64["dhhh"][:, 0, :, 1].sum(1)
    assert np.all(np.abs(g["logl"] - g64["logl"]) <= 1e-11 * sc)


def test_mixed_batch_invariance_and_entry_points(oracle_mod, Lb):
    """Bitwise batch invariance in mixed precision; a plan gives the direct call's bits; the
    gradient's log L agrees with the mixed forward's; the FP64-only Fisher entry point rejects
    the flag."""
    import torch
    T = 2.0 ** 17
    k0, nb = W.grid(T)
    od = H.oracle_detector(oracle_mod, W.LISA, T, k0, nb, _th_small(T), W.MODE_ALL, 4)
    gd = H.library_detector(Lb, od)
    th = W.draw_prior(40, 5, T)
    m = W.MODE_ALL | MIX
    full = Lb.loglike([gd], th, m, dhhh=True)
    perm = np.random.Generator(np.random.PCG64(1)).permutation(40)
    part = Lb.loglike([gd], th[perm[:13]], m, dhhh=True)
    assert np.array_equal(part["logl"], full["logl"][perm[:13]])
    assert np.array_equal(part["dhhh"], full["dhhh"][perm[:13]])
    tt = torch.tensor(th, device="cuda")
    pl = Lb.Plan([gd], 40, m, theta=tt, dhhh=True, autotune=False)
    pl.launch()
    torch.cuda.synchronize()
    assert np.array_equal(pl.logl.cpu().numpy(), full["logl"])
    pl.close()
    # the gradient takes the flag (tests/test_gpu_grad.py); its log L (per-bin sums in FP64 over
    # 128-bin tiles) agrees with the mixed forward's (double-word sums over 512-bin tiles)
    g = Lb.loglike_grad([gd], th[:2], m)
    np.testing.assert_allclose(g["logl"], full["logl"][:2], rtol=1e-12, atol=0)
    with pytest.raises(Lb.PeError) as e:
        Lb.fisher([gd], th[:2], m)
    assert e.value.status == Lb.PE_EINVAL
