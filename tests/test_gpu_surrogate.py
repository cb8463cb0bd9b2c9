"""The learned waveform surrogate: BF16 tensor-core MLP kernels against a CPU reference network,
the node-spline response path against the oracle, training on the GPU with the library's own
kernels, held-out mismatch against the plain generator (App. A's mismatch without the
maximisation), the fallback, the measured gain over the plain path, and the checkpoint."""
import math
import os

import numpy as np
import pytest

from paper_2602_12011_gb300 import workloads as W
from tests import _helpers as H

pytestmark = pytest.mark.gpu

T22 = 2.0 ** 22


@pytest.fixture(scope="module")
def Lb():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_2602_12011_gb300 import build as B
    from paper_2602_12011_gb300 import _lib
    B.build()
    return _lib


@pytest.fixture(scope="module")
def lisa22(Lb):
    k0, nb = W.grid(T22)
    d = Lb.Detector(W.LISA, T22, k0, nb)
    d.inject(W.theta_injection(T22), W.MODE_ALL, W.normals(nb, W.SEED_NOISE_SINGLE))
    return d


@pytest.fixture(scope="module")
def trained(Lb):
    """Trained once per module: 2^20 prior samples (seed 2605), 60 epochs, batch 1024."""
    import torch
    s = Lb.Surrogate(seed=2605)
    th = torch.tensor(W.draw_prior(1 << 20, 2605, T22), device="cuda")
    loss, curve = s.train(th, 60, batch=1024, lr=2e-3)
    assert np.all(np.isfinite(curve)) and curve[-1] < 0.05 * curve[0]
    return s


def test_mlp_kernels_match_reference_network(Lb):
    from oracle import mlp_ref
    s = Lb.Surrogate(seed=11)
    rng = np.random.default_rng(3)
    x = np.zeros((128, 64), np.float32)
    x[:, :11] = rng.standard_normal((128, 11))
    dy = (rng.standard_normal((128, 2560)) * 1e-3).astype(np.float32)
    y, g = s.mlp_debug(x, dy)
    yr, gr = mlp_ref.forward_backward(s.weights(), x, dy)
    assert np.linalg.norm(y - yr) / np.linalg.norm(yr) < 1e-3
    o = 0
    for i, n in zip(mlp_ref.DIMS[:-1], mlp_ref.DIMS[1:]):
        for size in (i * n, n):
            a, b = g[o:o + size], gr[o:o + size]
            o += size
            assert np.linalg.norm(a - b) / np.linalg.norm(b) < 5e-3
    s.close()


def test_node_spline_path_matches_oracle(oracle_mod, Lb):
    """With the plain generator's own node values (no network), the node-spline log-likelihood
    agrees with the oracle to the spline's accuracy."""
    import torch
    T = 2.0 ** 20
    k0, nb = W.grid(T)
    inj = np.array([2e6, 3.0, 0.5, 0.3, 25.8, 0.4, 1.3, 1.375, -1.2108, 2.659, 0.8 * T])
    od = H.oracle_detector(oracle_mod, W.LISA, T, k0, nb, inj, W.MODE_ALL, 5)
    gd = H.library_detector(Lb, od)
    s = Lb.Surrogate(seed=1)
    s.set_node_source(1)
    th = np.vstack([inj, W.draw_prior(6, 31, T)])
    th[1:, 0] = np.linspace(5e5, 9e6, 6)
    th[1:, 1] = np.minimum(th[1:, 1], 8.0)
    ll, used = s.loglike([gd], torch.tensor(th, device="cuda"), W.MODE_ALL)
    ll = ll.cpu().numpy()
    assert np.all(used.cpu().numpy() == 1)
    ref, dhhh = oracle_mod.loglike_batch([od], th, W.MODE_ALL)
    dd = od_dd = oracle_mod.loglike([od], inj, 0)["dd"].sum()
    for i in range(th.shape[0]):
        scale = 0.5 * dd + abs(dhhh[i, :, :, 0].sum()) + 0.5 * dhhh[i, :, :, 1].sum()
        assert abs(ll[i] - ref[i]) <= 1e-6 * scale, (i, ll[i], ref[i])
    s.close()


def test_heldout_mismatch_acceptance(Lb, lisa22, trained):
    """>= 99% of held-out samples inside the training box have mismatch <= 1e-3 against the plain
    generator on the 2^22 s LISA grid (noise-weighted inner product)."""
    import torch
    th = W.draw_prior(2048, 2606, T22)
    mm = trained.mismatch(lisa22, torch.tensor(th, device="cuda"), W.MODE_ALL).cpu().numpy()
    inbox = (th[:, 0] >= 3e5) & (th[:, 1] <= 8.0)
    assert inbox.mean() > 0.7
    assert np.all(mm[~inbox] == 0.0)                 # fallback samples are the plain signal
    frac = np.mean(mm[inbox] <= 1e-3)
    assert frac >= 0.99, (frac, np.quantile(mm[inbox], [0.5, 0.99]))


def test_fallback_is_the_plain_path_bitwise(Lb, lisa22, trained):
    import torch
    th = W.draw_prior(64, 2607, T22)
    th[::2, 1] = 9.5                                   # outside the box (q > 8)
    th[1::4, 0] = 2e5                                  # outside the box (light)
    tt = torch.tensor(th, device="cuda")
    ll, used = trained.loglike([lisa22], tt, W.MODE_ALL)
    ref = Lb.loglike([lisa22], th, W.MODE_ALL)["logl"]
    out = (th[:, 1] > 8.0) | (th[:, 0] < 3e5)
    assert np.array_equal(used.cpu().numpy(), (~out).astype(np.int32))
    assert np.array_equal(ll.cpu().numpy()[out], ref[out])


def test_surrogate_gain_over_plain_path(Lb, lisa22, trained):
    """What the trained network buys: the surrogate path against the plain per-bin path on the
    same in-box batch (1024 samples, 5 modes, 2^22 s), device-timed, median of five."""
    import torch
    th = W.draw_prior(1024, 2608, T22)
    th[:, 1] = np.minimum(th[:, 1], 8.0)
    th[:, 0] = np.maximum(th[:, 0], 3e5)
    tt = torch.tensor(th, device="cuda")
    out = torch.empty(1024, dtype=torch.float64, device="cuda")
    st = torch.cuda.current_stream()

    def plain():
        Lb.pe_loglike_batch([lisa22.handle], tt, 1024, W.MODE_ALL, out, None, None, st)

    def sur():
        trained.loglike([lisa22], tt, W.MODE_ALL)

    def med(fn):
        fn()
        ts = []
        for _ in range(5):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(st)
            fn()
            e1.record(st)
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1))
        return float(np.median(ts))

    tp, ts = med(plain), med(sur)
    print("plain %.2f ms, surrogate %.2f ms, gain %.2fx" % (tp, ts, tp / ts))
    assert tp / ts > 1.3


def test_checkpoint_roundtrip_and_corruption(Lb, trained, tmp_path):
    import torch
    path = str(tmp_path / "sur.bin")
    trained.save(path)
    s2 = Lb.Surrogate(seed=99)
    s2.load(path)
    th = torch.tensor(W.draw_prior(128, 5, T22), device="cuda")
    assert torch.equal(trained.predict(th), s2.predict(th))
    raw = bytearray(open(path, "rb").read())
    raw[100] ^= 0xFF
    bad = str(tmp_path / "bad.bin")
    open(bad, "wb").write(bytes(raw))
    with pytest.raises(Lb.PeError) as e:
        s2.load(bad)
    assert e.value.status == Lb.PE_EINVAL and "checksum" in str(e.value)
    s2.close()
