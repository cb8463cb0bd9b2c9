"""The seeded synthetic inputs (paper_2602_12011_gb300/workloads.py) follow the stated recipe: the
frequency grids of the three observation spans, the prior of the batched workloads, the
single-source injection and the noise draws; every generator is deterministic in its seed."""
import math

import numpy as np

from paper_2602_12011_gb300 import workloads as W


def test_grids_of_the_three_spans():
    # bins f_k = k/T inside [1e-4, 0.05] Hz
    for T, nb in ((2.0 ** 20, 52324), (2.0 ** 21, 104648), (2.0 ** 22, 209296)):
        k0, n = W.grid(T)
        assert n == nb
        assert k0 / T >= 1e-4 > (k0 - 1) / T
        assert (k0 + n - 1) / T <= 0.05 < (k0 + n) / T


def test_prior_draws_follow_the_recipe():
    T = 2.0 ** 22
    th = W.draw_prior(20000, 7, T)
    assert np.array_equal(th, W.draw_prior(20000, 7, T))
    assert not np.array_equal(th, W.draw_prior(20000, 8, T))
    lo = np.array([1e5, 1.0, -0.99, -0.99, 1.0, 0.0, 0.0, 0.0, -math.pi / 2, 0.0, 0.75 * T])
    hi = np.array([1e7, 10.0, 0.99, 0.99, 50.0, math.pi, 2 * math.pi, 2 * math.pi, math.pi / 2, math.pi, 0.85 * T])
    assert np.all(th >= lo) and np.all(th <= hi)
    # isotropic orientation and sky: cos(iota) and sin(beta) uniform on [-1, 1] (mean 0, var 1/3)
    for u in (np.cos(th[:, 5]), np.sin(th[:, 8])):
        assert abs(u.mean()) < 0.02 and abs(u.var() - 1.0 / 3.0) < 0.02
    # the uniform parameters fill their ranges (mean at the centre)
    for i in (0, 1, 2, 3, 4, 6, 7, 9, 10):
        assert abs(th[:, i].mean() - 0.5 * (lo[i] + hi[i])) < 0.02 * (hi[i] - lo[i])


def test_named_workloads():
    wl = W.batch_hm(1024)
    assert wl["name"] == "lisa_hm_T2^22_B1024" and wl["theta"].shape == (1024, 11)
    assert wl["mode_mask"] == W.MODE_ALL and wl["dets"][0][0]["name"] == "LISA"
    assert np.array_equal(wl["theta"], W.draw_prior(1024, W.SEED_BATCH_HM, 2.0 ** 22))
    net = W.network_hm(4096)
    assert [d[0]["name"] for d in net["dets"]] == ["LISA", "Taiji", "TianQin"]
    assert [d[1] for d in net["dets"]] == [2.0 ** 22, 2.0 ** 21, 2.0 ** 20]
    assert np.all(net["theta"][:, 10] < 2.0 ** 20)          # t_c inside every span
    inj = W.theta_injection(2.0 ** 20)
    assert inj[10] == 0.8 * 2.0 ** 20 and inj[0] == 1e6 and inj[1] == 2.0


def test_noise_draws():
    n = W.normals(50000, 3)
    assert n.shape == (3, 50000, 2)
    assert np.array_equal(n, W.normals(50000, 3))
    assert abs(n.mean()) < 0.01 and abs(n.var() - 1.0) < 0.01
