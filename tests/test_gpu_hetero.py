"""GPU parity of the heterodyned (relative-binning) likelihood (pe_hetero_*), the heterodyning idea
of Sec. 1, against the oracle's plain implementation (oracle/hetero.py) on the same data, reference,
edges and samples. Also checks it against the library's exact likelihood, where it is exact (at the
reference; for d_L and phi_c changes) and near it (Fisher-Gaussian posterior draws of the full
workload)."""
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


def _near(th0, n, seed, scale):
    g = np.random.Generator(np.random.PCG64(seed))
    d = np.array([2e3, 0.01, 0.01, 0.01, 0.3, 0.01, 0.05, 1e-3, 1e-3, 0.01, 20.0]) * scale
    th = th0[None, :] + g.standard_normal((n, 11)) * d[None, :]
    th[:, 2:4] = np.clip(th[:, 2:4], -0.98, 0.98)
    return th


@pytest.mark.parametrize("mix", [False, True], ids=["fp64", "mixed"])
@pytest.mark.parametrize("det", [W.LISA, W.TIANQIN], ids=["lisa", "tianqin"])
def test_hetero_parity_with_oracle(oracle_mod, Lb, det, mix):
    from oracle import hetero as HT
    T = 2.0 ** 18
    k0, nb = W.grid(T)
    th0 = np.array([8e5, 2.0, 0.4, -0.2, 20.0, 0.6, 0.9, 2.0, 0.4, 1.1, 0.8 * T])
    od = H.oracle_detector(oracle_mod, det, T, k0, nb, th0, W.MODE_ALL, 19)
    gd = H.library_detector(Lb, od)
    edges = HT.default_edges(T, k0, nb, th0, W.MODE_ALL, 64)
    oh = HT.Hetero(od, th0, W.MODE_ALL, edges)
    gh = Lb.Hetero(gd, th0, W.MODE_ALL | (Lb.PE_PREC_MIXED if mix else 0), edges=edges)
    th = np.vstack([th0, _near(th0, 12, 5, 1.0)])
    g = Lb.hetero_loglike([gh], th, dhhh=True)
    Q = H.floor_terms(oracle_mod, [od], th, W.MODE_ALL)
    for s in range(th.shape[0]):
        r = oh.loglike(th[s])
        sc = 0.5 * r["dd"].sum() + abs(r["dh"].sum()) + 0.5 * r["hh"].sum()
        assert abs(g["logl"][s] - r["logl"]) <= 1e-10 * sc, (s, g["logl"][s], r["logl"])
        H.assert_loglike_parity({"logl": g["logl"][s:s + 1], "dhhh": g["dhhh"][s:s + 1]}, np.array([r["logl"]]),
                                np.stack([r["dh"], r["hh"]], -1)[None, None], r["dd"], Q[s],
                                u=H.U_DW if mix else H.U64, name="hetero:%s:%s" % (det["name"], mix))
    gh.close()


@pytest.mark.parametrize("mix", [False, True], ids=["fp64", "mixed"])
def test_hetero_network_parity(oracle_mod, Lb, mix):
    from oracle import hetero as HT
    Ts = (2.0 ** 18, 2.0 ** 17, 2.0 ** 16)
    th0 = np.array([6e5, 3.0, 0.2, 0.5, 12.0, 1.1, 0.3, 4.0, -0.6, 0.4, 0.8 * 2.0 ** 16])
    ohs, ghs, gds = [], [], []
    for det, T in zip((W.LISA, W.TAIJI, W.TIANQIN), Ts):
        k0, nb = W.grid(T)
        od = H.oracle_detector(oracle_mod, det, T, k0, nb, th0, W.MODE_ALL, 23)
        gd = H.library_detector(Lb, od)
        e = HT.default_edges(T, k0, nb, th0, W.MODE_ALL, 48)
        ohs.append(HT.Hetero(od, th0, W.MODE_ALL, e))
        gds.append(gd)
        ghs.append(Lb.Hetero(gd, th0, W.MODE_ALL | (Lb.PE_PREC_MIXED if mix else 0), edges=e))
    th = np.vstack([th0, _near(th0, 6, 7, 1.0)])
    g = Lb.hetero_loglike(ghs, th, dhhh=True)
    Q = H.floor_terms(oracle_mod, [o.odet for o in ohs], th, W.MODE_ALL)
    for s in range(th.shape[0]):
        r = HT.loglike_network(ohs, th[s])
        sc = 0.5 * r["dd"].sum() + abs(r["dh"].sum()) + 0.5 * r["hh"].sum()
        assert abs(g["logl"][s] - r["logl"]) <= 1e-10 * sc
        H.assert_loglike_parity({"logl": g["logl"][s:s + 1], "dhhh": g["dhhh"][s:s + 1]}, np.array([r["logl"]]),
                                np.stack([r["dh"], r["hh"]], -1)[None], r["dd"], Q[s],
                                u=H.U_DW if mix else H.U64, name="hetero_network:%s" % mix)


def test_hetero_against_exact_likelihood(Lb):
    """Full workload (LISA, 5 modes, 2^22 s): exact at the reference and for d_L, phi_c changes;
    within a few 1e-2 in log L for draws in the posterior's bulk (256 coarse bins)."""
    import torch
    wl = W.batch_hm(64)
    det, T, k0, nb = wl["dets"][0]
    g = Lb.Detector(det, T, k0, nb)
    g.inject(wl["inj"], wl["inj_mask"], W.normals(nb, wl["noise_seed"]))
    th0 = wl["inj"]
    het = Lb.Hetero(g, th0, W.MODE_ALL, nbins_coarse=256)
    hetm = Lb.Hetero(g, th0, W.MODE_ALL | Lb.PE_PREC_MIXED, nbins_coarse=256)
    cases = np.vstack([th0, th0 * np.r_[1, 1, 1, 1, 1.2, 1, 1, 1, 1, 1, 1], th0 + np.r_[0, 0, 0, 0, 0, 0, 0.4, 0, 0, 0, 0]])
    ex = Lb.loglike([g], cases, W.MODE_ALL, dhhh=True)
    ht = Lb.hetero_loglike([het], cases)
    sc = 0.5 * g.data_norm().sum() + np.abs(ex["dhhh"][:, 0, :, 0].sum(1)) + 0.5 * ex["dhhh"][:, 0, :, 1].sum(1)
    assert np.all(np.abs(ht["logl"] - ex["logl"]) <= 1e-10 * sc)
    # draws around the injection: the all-parameter Fisher-Gaussian is far wider than the true
    # posterior here (its unit draws cost ~1e3 in log L), so take its 0.1-scaled draws (median
    # log L change -0.7, the posterior's bulk) and 0.3-scaled ones kept where log L drops < 50
    idx = np.arange(11, dtype=np.int32)
    ex0 = Lb.loglike([g], th0[None, :], W.MODE_ALL)["logl"][0]
    for zs, bound in ((0.1, 0.05), (0.3, 0.15)):
        nrm = zs * np.random.Generator(np.random.PCG64(31)).standard_normal((256, 11))
        _, draws = Lb.fisher_gaussian([g], th0, W.MODE_ALL, idx, nrm)
        ok = (draws[:, 1] >= 1.0) & (np.abs(draws[:, 2]) < 1) & (np.abs(draws[:, 3]) < 1) & (draws[:, 4] > 0)
        tt = torch.tensor(draws[ok], device="cuda")
        ex = Lb.loglike([g], tt, W.MODE_ALL)["logl"].cpu().numpy()
        ht = Lb.hetero_loglike([het], tt)["logl"].cpu().numpy()
        assert np.all(np.isfinite(ht))
        near = ex - ex0 > -50.0
        assert near.sum() > 100
        # measured at 256 bins: 6.5e-3 (0.1-scaled), 3.0e-2 (0.3-scaled, within 50 of the peak)
        assert np.abs(ht - ex)[near].max() < bound, np.abs(ht - ex)[near].max()
        # the mixed-precision edge evaluation changes the heterodyned log L by rounding only
        hm = Lb.hetero_loglike([hetm], tt)["logl"].cpu().numpy()
        assert np.all(np.abs(hm - ht) <= 1e-11 * (np.abs(ht) + 0.5 * g.data_norm().sum()))
    het.close()
    hetm.close()


def test_hetero_errors(Lb):
    T = 2.0 ** 16
    k0, nb = W.grid(T)
    d = Lb.Detector(W.LISA, T, k0, nb)
    th0 = W.theta_injection(T)
    with pytest.raises(Lb.PeError) as e:
        Lb.Hetero(d, th0, W.MODE_ALL, edges=np.array([0, 5]))          # no data yet
    assert e.value.status == Lb.PE_ESTATE
    d.set_data(np.zeros((3, nb), dtype=np.complex128))
    with pytest.raises(Lb.PeError) as e:
        Lb.Hetero(d, th0, W.MODE_ALL, edges=np.array([0, 5, 5]))
    assert e.value.status == Lb.PE_EINVAL
    with pytest.raises(Lb.PeError) as e:
        Lb.Hetero(d, th0, W.MODE_ALL, edges=np.arange(700))
    assert e.value.status == Lb.PE_EINVAL
    with pytest.raises(Lb.PeError) as e:
        Lb.Hetero(d, th0, W.MODE_ALL | Lb.PE_PREC_FP32, edges=np.array([0, 40, 90]))
    assert e.value.status == Lb.PE_EINVAL
    a = Lb.Hetero(d, th0, W.MODE_ALL, edges=np.array([0, 40, 90]))
    b = Lb.Hetero(d, th0, W.MODE_22, edges=np.array([0, 40, 90]))
    with pytest.raises(Lb.PeError) as e:
        Lb.hetero_loglike([a, b], th0[None, :])
    assert e.value.status == Lb.PE_EINVAL
