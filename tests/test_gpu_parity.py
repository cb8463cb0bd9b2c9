"""GPU parity of the CUDA path (through the C ABI) against the FP64 CPU oracle.

Element by element on identical seeded inputs: the per-bin A/E/T signal, the PSD, and per
sample log L with <d|h>, <h|h> per detector and channel, to a relative 1e-10 of the
likelihood's scale (Eq. eq_ll_fd). Sizes span several 128-bin tiles with a ragged tail, and
the full single-detector higher-mode workload (T = 2^22 s, B = 1024) is checked on sampled
outputs in the same launch configuration the benchmark times.
"""
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
    _lib.lib()
    return _lib


def _th_small(T):
    return np.array([1e6, 2.0, 0.5, 0.3, 25.8, 0.4, 1.3, 1.375, -1.2108, 2.659, 0.8 * T])


@pytest.mark.parametrize("det", [W.LISA, W.TAIJI, W.TIANQIN, dict(W.LISA, tdi_gen=15)], ids=["lisa", "taiji",
                                                                                              "tianqin", "lisa15"])
def test_psd_model_parity(oracle_mod, Lb, det):
    T = 2.0 ** 20
    k0, nb = W.grid(T)
    d = Lb.Detector(det, T, k0, nb)
    np.testing.assert_allclose(d.psd(), oracle_mod.psd(det, H.grid_f(T, k0, nb)), rtol=1e-12)


@pytest.mark.parametrize("det", [W.LISA, W.TAIJI, W.TIANQIN, dict(W.LISA, tdi_gen=15)], ids=["lisa", "taiji",
                                                                                              "tianqin", "lisa15"])
@pytest.mark.parametrize("mask", [W.MODE_22, W.MODE_ALL, 0x02, 0x04, 0x08, 0x10])
def test_signal_parity_per_bin(oracle_mod, Lb, det, mask):
    """Every bin of the A/E/T signal (rows A1-A6) against the oracle's direct evaluation."""
    T = 2.0 ** 18
    k0, nb = W.grid(T)
    th = _th_small(T)
    th[0] = 3e5
    d = Lb.Detector(det, T, k0, nb)
    h = d.signal(th, mask)
    ref = oracle_mod.response(det, th, mask, H.grid_f(T, k0, nb))
    phi = H.phase_magnitude(oracle_mod, th, mask, H.grid_f(T, k0, nb))
    H.assert_signal_parity(h, ref, "signal_per_bin:%s:%s:%#x" % (det["name"], det["tdi_gen"], mask), phi)


def test_injection_parity(oracle_mod, Lb):
    """pe_inject (signal + noise scaled by the library PSD) against the oracle's data."""
    T = 2.0 ** 18
    k0, nb = W.grid(T)
    th = _th_small(T)
    nrm = W.normals(nb, 5)
    d = Lb.Detector(W.LISA, T, k0, nb)
    d.inject(th, W.MODE_ALL, nrm)
    ref = oracle_mod.make_data(W.LISA, th, W.MODE_ALL, T, k0, nb, nrm)
    psd = oracle_mod.psd(W.LISA, H.grid_f(T, k0, nb))
    od = oracle_mod.Detector(W.LISA, T, k0, nb, ref, psd)
    r = oracle_mod.loglike([od], th, 0)                 # mode mask 0: h = 0, gives <d|d>
    np.testing.assert_allclose(d.data_norm(), r["dd"][0], rtol=1e-11)


def test_loglike_single_source_full_grid(oracle_mod, Lb):
    """Plain single-source path: LISA, (2,2), T = 2^20 s (52,324 bins), noisy data."""
    wl = W.single_22()
    det, T, k0, nb = wl["dets"][0]
    od = H.oracle_detector(oracle_mod, det, T, k0, nb, wl["inj"], wl["inj_mask"], wl["noise_seed"])
    gd = H.library_detector(Lb, od)
    th = np.vstack([wl["inj"], wl["inj"] + np.array([1e2, 1e-3, 0, 0, 0.1, 0.01, 0.1, 1e-3, 1e-3, 0.01, 5.0])])
    g = Lb.loglike([gd], th, wl["mode_mask"], dhhh=True)
    ll, dhhh = oracle_mod.loglike_batch([od], th, wl["mode_mask"])
    H.assert_loglike_parity(g, ll, dhhh, od_dd(oracle_mod, od), H.floor_terms(oracle_mod, [od], th, wl["mode_mask"]))
    np.testing.assert_allclose(gd.data_norm(), od_dd(oracle_mod, od)[0], rtol=1e-12)


def od_dd(O, od):
    r = O.loglike([od], np.array([1e6, 2, 0, 0, 1, 0, 0, 0, 0, 0, 0.0]), 0)
    return r["dd"]


@pytest.mark.parametrize("T,nbad", [(2.0 ** 14, 0), (2.0 ** 17, 3)])
def test_loglike_batch_hm_small_grids(oracle_mod, Lb, T, nbad):
    """Higher modes on grids of several tiles with a ragged tail, prior samples; out-of-domain
    samples get -inf and the status bit, the rest are unaffected."""
    k0, nb = W.grid(T)
    assert nb % 128 != 0
    od = H.oracle_detector(oracle_mod, W.LISA, T, k0, nb, _th_small(T), W.MODE_ALL, 11)
    gd = H.library_detector(Lb, od)
    th = W.draw_prior(24, 77, T)
    th[:, 0] = np.geomspace(1e5, 1e7, 24)
    for i in range(nbad):
        th[3 * i + 1, [1, 2, 4][i]] = [0.5, 1.2, -1.0][i]
    g = Lb.loglike([gd], th, W.MODE_ALL, dhhh=True, status=True)
    ll, dhhh = oracle_mod.loglike_batch([od], th, W.MODE_ALL)
    bad = g["status"] != 0
    assert bad.sum() == nbad
    assert np.all(np.isneginf(g["logl"][bad]))
    good = ~bad
    H.assert_loglike_parity({"logl": g["logl"][good], "dhhh": g["dhhh"][good]}, ll[good], dhhh[good],
                            od_dd(oracle_mod, od), H.floor_terms(oracle_mod, [od], th[good], W.MODE_ALL))


def test_loglike_edge_grids(oracle_mod, Lb):
    """One-bin grid, a grid of exactly one tile, and a grid where no bin is active."""
    T = 2.0 ** 16
    for k0, nb in ((700, 1), (100, 128), (3000, 37)):
        od = H.oracle_detector(oracle_mod, W.LISA, T, k0, nb, _th_small(T), W.MODE_ALL, 3)
        gd = H.library_detector(Lb, od)
        th = np.vstack([_th_small(T), _th_small(T)])
        th[1, 0] = 1e5
        g = Lb.loglike([gd], th, W.MODE_ALL, dhhh=True)
        ll, dhhh = oracle_mod.loglike_batch([od], th, W.MODE_ALL)
        H.assert_loglike_parity(g, ll, dhhh, od_dd(oracle_mod, od), H.floor_terms(oracle_mod, [od], th, W.MODE_ALL))


def test_maximum_batch_and_detector_count(oracle_mod, Lb):
    """The largest batch the entry points take (B = 2^20, on a small ragged grid) and the largest
    detector count (8 handles): sampled outputs against the oracle, bitwise equality with a small
    batch of the same samples, and PE_EINVAL one past each limit."""
    import torch
    T = 2.0 ** 14
    k0, nb = W.grid(T)
    od = H.oracle_detector(oracle_mod, W.LISA, T, k0, nb, _th_small(T), W.MODE_ALL, 5)
    gd = H.library_detector(Lb, od)
    B = 1 << 20
    th = W.draw_prior(B, 91, T)
    tt = torch.tensor(th, device="cuda")
    g = Lb.loglike([gd], tt, W.MODE_ALL, dhhh=True)
    out, dh = g["logl"].cpu().numpy(), g["dhhh"].cpu().numpy()
    del g, tt
    assert np.all(np.isfinite(out))
    pick = np.r_[0, 1, B // 2, B - 1, np.random.Generator(np.random.PCG64(3)).choice(B, 6, replace=False)]
    ll, dhhh = oracle_mod.loglike_batch([od], th[pick], W.MODE_ALL)
    H.assert_loglike_parity({"logl": out[pick], "dhhh": dh[pick]}, ll, dhhh, od_dd(oracle_mod, od),
                            H.floor_terms(oracle_mod, [od], th[pick], W.MODE_ALL))
    small = Lb.loglike([gd], th[pick], W.MODE_ALL)
    assert np.array_equal(small["logl"], out[pick])
    with pytest.raises(Lb.PeError) as e:
        Lb.loglike([gd], np.vstack([th[:1]] * (B + 1)), W.MODE_ALL)
    assert e.value.status == Lb.PE_EINVAL
    del th
    # eight detectors: LISA, Taiji and TianQin-like grids, repeated with other noise draws
    dets = [(W.LISA, 2.0 ** 14), (W.TAIJI, 2.0 ** 14), (W.TIANQIN, 2.0 ** 14), (W.LISA, 2.0 ** 13),
            (W.TAIJI, 2.0 ** 13), (W.TIANQIN, 2.0 ** 13), (dict(W.LISA, tdi_gen=15), 2.0 ** 14), (W.LISA, 2.0 ** 15)]
    ods, gds = [], []
    for i, (det, Ti) in enumerate(dets):
        k0i, nbi = W.grid(Ti)
        o = H.oracle_detector(oracle_mod, det, Ti, k0i, nbi, _th_small(2.0 ** 13), W.MODE_ALL, 40 + i)
        ods.append(o)
        gds.append(H.library_detector(Lb, o))
    th8 = np.vstack([_th_small(2.0 ** 13), W.draw_prior(7, 92, 2.0 ** 13)])
    g8 = Lb.loglike(gds, th8, W.MODE_ALL, dhhh=True)
    ll8, dhhh8 = oracle_mod.loglike_batch(ods, th8, W.MODE_ALL)
    dd8 = np.array([od_dd(oracle_mod, o) for o in ods])
    H.assert_loglike_parity(g8, ll8, dhhh8, dd8, H.floor_terms(oracle_mod, ods, th8, W.MODE_ALL))
    with pytest.raises(Lb.PeError) as e:
        Lb.loglike(gds + gds[:1], th8, W.MODE_ALL)
    assert e.value.status == Lb.PE_EINVAL


def test_network_parity(oracle_mod, Lb):
    """LISA + Taiji + TianQin with uneven grids (smaller spans for the oracle's speed)."""
    Ts = (2.0 ** 19, 2.0 ** 18, 2.0 ** 17)
    ods, gds = [], []
    inj = _th_small(2.0 ** 17)
    for det, T in zip((W.LISA, W.TAIJI, W.TIANQIN), Ts):
        k0, nb = W.grid(T)
        od = H.oracle_detector(oracle_mod, det, T, k0, nb, inj, W.MODE_ALL, 21)
        ods.append(od)
        gds.append(H.library_detector(Lb, od))
    th = W.draw_prior(6, 99, 2.0 ** 17)
    th = np.vstack([inj, th])
    g = Lb.loglike(gds, th, W.MODE_ALL, dhhh=True)
    ll, dhhh = oracle_mod.loglike_batch(ods, th, W.MODE_ALL)
    dd = np.array([od_dd(oracle_mod, od)[0] for od in ods])
    H.assert_loglike_parity(g, ll, dhhh, dd, H.floor_terms(oracle_mod, ods, th, W.MODE_ALL))


def test_batch_invariance_bitwise(oracle_mod, Lb):
    """A sample's result depends only on its own theta: identical bits in any batch."""
    T = 2.0 ** 17
    k0, nb = W.grid(T)
    od = H.oracle_detector(oracle_mod, W.LISA, T, k0, nb, _th_small(T), W.MODE_ALL, 4)
    gd = H.library_detector(Lb, od)
    th = W.draw_prior(40, 5, T)
    full = Lb.loglike([gd], th, W.MODE_ALL, dhhh=True)
    perm = np.random.Generator(np.random.PCG64(1)).permutation(40)
    part = Lb.loglike([gd], th[perm[:13]], W.MODE_ALL, dhhh=True)
    assert np.array_equal(part["logl"], full["logl"][perm[:13]])
    assert np.array_equal(part["dhhh"], full["dhhh"][perm[:13]])
    for i in (0, 17, 39):
        one = Lb.loglike([gd], th[i:i + 1], W.MODE_ALL)
        assert one["logl"][0] == full["logl"][i]


def test_device_pointers_and_stream(oracle_mod, Lb):
    """torch CUDA tensors in and out, on a side stream, equal the host-buffer path bit for bit."""
    import torch
    T = 2.0 ** 16
    k0, nb = W.grid(T)
    od = H.oracle_detector(oracle_mod, W.LISA, T, k0, nb, _th_small(T), W.MODE_ALL, 8)
    gd = H.library_detector(Lb, od)
    th = W.draw_prior(9, 6, T)
    host = Lb.loglike([gd], th, W.MODE_ALL, dhhh=True)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        tt = torch.tensor(th, device="cuda")
        dev = Lb.loglike([gd], tt, W.MODE_ALL, dhhh=True, stream=s)
    s.synchronize()
    assert np.array_equal(dev["logl"].cpu().numpy(), host["logl"])
    assert np.array_equal(dev["dhhh"].cpu().numpy(), host["dhhh"])


def test_errors_are_status_codes(Lb):
    d = Lb.Detector(W.LISA, 2.0 ** 16, *W.grid(2.0 ** 16))
    with pytest.raises(Lb.PeError) as e:
        Lb.loglike([d], W.draw_prior(2, 1, 2.0 ** 16), W.MODE_ALL)
    assert e.value.status == Lb.PE_ESTATE
    d.set_data(np.zeros((3, d.nb), dtype=np.complex128))
    with pytest.raises(Lb.PeError) as e:
        Lb.loglike([d], W.draw_prior(2, 1, 2.0 ** 16), 0x40)
    assert e.value.status == Lb.PE_EINVAL
    bad = d.psd()
    bad[1, 5] = 0.0
    with pytest.raises(Lb.PeError) as e:
        d.set_data(np.zeros((3, d.nb), dtype=np.complex128), bad)
    assert e.value.status == Lb.PE_EINVAL


def test_full_size_hm_batch_sampled(oracle_mod, Lb):
    """The benchmark's workload and launch: LISA, 5 modes, T = 2^22 s (209,296 bins), B = 1024,
    one batched call; a spread of 16 samples is checked against the oracle."""
    wl = W.batch_hm(1024)
    det, T, k0, nb = wl["dets"][0]
    od = H.oracle_detector(oracle_mod, det, T, k0, nb, wl["inj"], wl["inj_mask"], wl["noise_seed"])
    gd = H.library_detector(Lb, od)
    th = wl["theta"]
    g = Lb.loglike([gd], th, wl["mode_mask"], dhhh=True)
    assert np.all(np.isfinite(g["logl"]))
    # 16 samples spread over the batch, biased to the cheap (heavy) ones for the oracle's speed,
    # plus the three lightest (longest in band)
    order = np.argsort(th[:, 0])
    pick = np.unique(np.r_[order[:3], order[np.linspace(200, 1023, 13).astype(int)]])
    ll, dhhh = oracle_mod.loglike_batch([od], th[pick], wl["mode_mask"])
    H.assert_loglike_parity({"logl": g["logl"][pick], "dhhh": g["dhhh"][pick]}, ll, dhhh, od_dd(oracle_mod, od),
                            H.floor_terms(oracle_mod, [od], th[pick], wl["mode_mask"]))
