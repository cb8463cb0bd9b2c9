"""Uneven batches (many samples, detectors and grid lengths in one persistent launch) through a
CUDA-graph plan with autotuned launch parameters: bit-identical to the direct call, and the
detector-network workload (LISA 2^22 s + Taiji 2^21 s + TianQin 2^20 s, B = 4096) against the
oracle on sampled outputs (Sec. 2.2 joint likelihood over detectors)."""
import os

import numpy as np
import pytest

from paper_2602_12011_gb300 import workloads as W
from tests import _helpers as H

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def Lb(tmp_path_factory):
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    os.environ["PE_TUNE_CACHE"] = str(tmp_path_factory.mktemp("tune") / "tune.json")
    from paper_2602_12011_gb300 import build as B
    from paper_2602_12011_gb300 import _lib
    B.build()
    return _lib


def _net(O, Lb, Ts, seed=21):
    inj = np.array([1e6, 2.0, 0.5, 0.3, 25.8, 0.4, 1.3, 1.375, -1.2108, 2.659, 0.8 * min(Ts)])
    ods, gds = [], []
    for det, T in zip((W.LISA, W.TAIJI, W.TIANQIN), Ts):
        k0, nb = W.grid(T)
        od = H.oracle_detector(O, det, T, k0, nb, inj, W.MODE_ALL, seed)
        ods.append(od)
        gds.append(H.library_detector(Lb, od))
    return inj, ods, gds


def test_plan_bitwise_equal_to_direct_call_and_refill(oracle_mod, Lb):
    import torch
    Ts = (2.0 ** 17, 2.0 ** 16, 2.0 ** 15)
    _, _, gds = _net(oracle_mod, Lb, Ts)
    B = 50
    th1 = W.draw_prior(B, 11, 2.0 ** 15)
    th2 = W.draw_prior(B, 12, 2.0 ** 15)
    theta = torch.tensor(th1, device="cuda")
    plan = Lb.Plan(gds, B, W.MODE_ALL, theta=theta, dhhh=True, autotune=True)
    info = plan.info()
    assert 0 <= info["fwd_variant"] <= 2 and info["ctas_per_sm"] in (2, 4, 8, 16)
    for th in (th1, th2, th1):
        theta.copy_(torch.tensor(th, device="cuda"))
        plan.launch()
        torch.cuda.synchronize()
        ref = Lb.loglike(gds, th, W.MODE_ALL, dhhh=True)
        assert np.array_equal(plan.logl.cpu().numpy(), ref["logl"])
        assert np.array_equal(plan.dhhh.cpu().numpy(), ref["dhhh"])
    plan.close()


def test_autotune_changes_no_result(oracle_mod, Lb):
    import torch
    T = 2.0 ** 17
    k0, nb = W.grid(T)
    d = Lb.Detector(W.LISA, T, k0, nb)
    d.inject(W.theta_injection(T), W.MODE_ALL, W.normals(nb, 2))
    th = W.draw_prior(77, 13, T)
    before = Lb.loglike([d], th, W.MODE_ALL, dhhh=True)
    choice = Lb.pe_autotune([d.handle], torch.tensor(th, device="cuda"), 77, W.MODE_ALL)
    assert choice["tuned_ms"] > 0
    after = Lb.loglike([d], th, W.MODE_ALL, dhhh=True)
    assert np.array_equal(before["logl"], after["logl"]) and np.array_equal(before["dhhh"], after["dhhh"])
    assert os.path.exists(os.environ["PE_TUNE_CACHE"])


@pytest.mark.parametrize("mix", [False, True], ids=["fp64", "mixed"])
def test_every_tuning_choice_gives_the_same_bits(oracle_mod, Lb, mix):
    """Work items of 1, 2, 4 and 8 sub-tiles, each register-budget variant and two grid sizes,
    recorded with pe_tune_set: the direct call and a plan give the same bits for every choice, on
    a detector network with uneven grids and a ragged tail."""
    import torch
    dets = []
    for det, T in ((W.LISA, 2.0 ** 16), (W.TAIJI, 2.0 ** 15), (W.TIANQIN, 2.0 ** 14)):
        k0, nb = W.grid(T)
        d = Lb.Detector(det, T, k0, nb)
        d.inject(W.theta_injection(2.0 ** 14), W.MODE_ALL, W.normals(nb, 5))
        dets.append(d)
    B = 37
    m = W.MODE_ALL | (Lb.PE_PREC_MIXED if mix else 0)
    th = W.draw_prior(B, 21, 2.0 ** 14)
    hs = [d.handle for d in dets]
    ref = None
    for r in (1, 2, 4, 8):
        for v, c in ((0, 16), (1, 2), (2, 8)):
            Lb.pe_tune_set(hs, B, m, v, c, r)
            out = Lb.loglike(dets, th, m, dhhh=True)
            tt = torch.tensor(th, device="cuda")
            pl = Lb.Plan(dets, B, m, theta=tt, dhhh=True, autotune=False)
            info = pl.info()
            assert (info["fwd_variant"], info["ctas_per_sm"], info["subtiles"]) == (v, c, r)
            pl.launch()
            torch.cuda.synchronize()
            if ref is None:
                ref = out
            assert np.array_equal(out["logl"], ref["logl"]) and np.array_equal(out["dhhh"], ref["dhhh"])
            assert np.array_equal(pl.logl.cpu().numpy(), ref["logl"])
            pl.close()
    with pytest.raises(Lb.PeError) as e:
        Lb.pe_tune_set(hs, B, m, 0, 8, 3)
    assert e.value.status == Lb.PE_EINVAL


def test_network_full_size_plan_sampled(oracle_mod, Lb):
    """Detector network at full spans (209,296 + 104,648 + 52,324 bins), B = 4096 in one graph
    launch; a spread of samples is checked against the oracle."""
    import torch
    wl = W.network_hm(4096)
    ods, gds = [], []
    for det, T, k0, nb in wl["dets"]:
        od = H.oracle_detector(oracle_mod, det, T, k0, nb, wl["inj"], wl["inj_mask"], wl["noise_seed"])
        ods.append(od)
        gds.append(H.library_detector(Lb, od))
    th = wl["theta"]
    plan = Lb.Plan(gds, th.shape[0], wl["mode_mask"], theta=torch.tensor(th, device="cuda"), dhhh=True)
    plan.launch()
    torch.cuda.synchronize()
    logl = plan.logl.cpu().numpy()
    dhhh = plan.dhhh.cpu().numpy()
    assert np.all(np.isfinite(logl))
    order = np.argsort(th[:, 0])
    pick = np.r_[order[-5:], order[len(order) // 2]]
    ll, ref = oracle_mod.loglike_batch(ods, th[pick], wl["mode_mask"])
    dd = np.array([oracle_mod.loglike([od], th[0], 0)["dd"][0] for od in ods])
    H.assert_loglike_parity({"logl": logl[pick], "dhhh": dhhh[pick]}, ll, ref, dd,
                            H.floor_terms(oracle_mod, ods, th[pick], wl["mode_mask"]))
    plan.close()
