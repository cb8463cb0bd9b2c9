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
# the default box of the spline path: Mtot in [1e5, 1e7] Msun, q <= 10, |chi| <= 0.99 (the prior's
# range), with the network's node values up to q = 8 and the plain generator's above
BOX_MLO, BOX_QMAX, NET_QMAX = 1e5, 10.0, 8.0


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


def _gemm_check(name, got, A, Bt, bias=None, rel=1e-5):
    """One dense layer's fp32 output against the exact (fp64) product of the kernel's own bf16
    operands, element by element. Every product of two bf16 values is exact in fp32, so the only
    error is the fp32 accumulation of K terms: at most (K + 2) 2^-23 sum_k |a_k b_k| (+ the same
    relative size of the bias), a bound that holds for round-to-nearest and for truncating
    accumulation alike. The bar is 1e-5 relative, with the floor of an fp32 sum: partial sums up
    to sum_k |a_k b_k| in size each round by up to half an fp32 ulp, so an element that cancels
    cannot be known better than a few 2^-24 sum_k |a_k b_k|; the floor is 4 x 2^-24 of it."""
    A = A.astype(np.float64)
    Bt = Bt.astype(np.float64)
    exact = A @ Bt.T
    absum = np.abs(A) @ np.abs(Bt).T
    if bias is not None:
        exact = exact + bias[None, :]
        absum = absum + np.abs(bias)[None, :]
    K = A.shape[1]
    err = np.abs(got.astype(np.float64) - exact)
    hard = (K + 2) * 2.0 ** -23 * absum
    assert np.all(err <= hard), (name, "accumulation bound", np.max(err / np.maximum(hard, 1e-300)))
    tol = np.maximum(rel * np.abs(exact), 4 * 2.0 ** -24 * absum)
    H.record_margin("mlp:" + name, np.max(err / np.maximum(tol, 1e-300)))
    assert np.all(err <= tol), (name, np.max(err / np.maximum(tol, 1e-300)))


def test_mlp_layers_elementwise_against_their_own_inputs(Lb):
    """Each tensor-core product of the forward and backward pass, and each elementwise stage,
    element by element against an exact recomputation from the kernels' own (bf16-rounded) inputs
    (pe_surrogate_mlp_trace): outputs and cotangents to 1e-5 (_gemm_check), the weight gradients
    to 1e-4; SiLU stores the round-to-nearest bf16 of its fp32 value (a ulp flip allowed where
    __expf's few-ulp error crosses a rounding midpoint, in under 0.1 % of elements); SiLU' to
    2e-6 relative; the bias gradients (fp32 column sums) to their summation bound."""
    s = Lb.Surrogate(seed=11)
    for B in (128, 192):          # one 128-row tile; a second, partial tile (rows past B zero-filled)
        _mlp_layers_check(Lb, s, B)
    s.close()


def _mlp_layers_check(Lb, s, B):
    from oracle import mlp_ref
    rng = np.random.default_rng(B)
    x = np.zeros((B, 64), np.float32)
    x[:, :11] = rng.standard_normal((B, 11))
    dy = (rng.standard_normal((B, 2560)) * 1e-3).astype(np.float32)
    y, g, tr = s.mlp_trace(x, dy)
    layers = mlp_ref.unpack(s.weights())
    bf = mlp_ref.bf16
    np.testing.assert_array_equal(tr["X"], bf(x))
    Hin = tr["X"]
    for l in range(3):
        W, b = layers[l]
        _gemm_check("Z%d" % l, tr["Z%d" % l], Hin, bf(W), b)
        Z = tr["Z%d" % l].astype(np.float64)
        ref = bf(Z / (1.0 + np.exp(-Z)))
        d = np.abs(tr["H%d" % l] - ref)
        ulp = np.abs(ref) * 2.0 ** -7 + 1e-38
        assert np.all(d <= ulp), ("H%d" % l, np.max(d / ulp))
        assert np.mean(d > 0) < 1e-3, ("H%d" % l, np.mean(d > 0))
        Hin = tr["H%d" % l]
    W3, b3 = layers[3]
    _gemm_check("Y", tr["Y"], Hin, bf(W3), b3)
    np.testing.assert_array_equal(tr["Y"], y)
    # backward: dH2 = bf16(dY) W3; per layer dZ = dH SiLU'(Z), gW = bf16(dZ)^T H_in, gb = sum dZ,
    # dH_{l-1} = bf16(dZ) W_l
    dYb = bf(dy)
    o, gw = 0, {}
    for l, (i, n) in enumerate(zip(mlp_ref.DIMS[:-1], mlp_ref.DIMS[1:])):
        gw[l] = (g[o:o + i * n].reshape(n, i), g[o + i * n:o + i * n + n])
        o += i * n + n
    _gemm_check("gW3", gw[3][0], dYb.T, tr["H2"].T, rel=1e-4)
    colsum_bound = lambda v: (v.shape[0] + 1) * 2.0 ** -24 * np.abs(v).sum(0)
    assert np.all(np.abs(gw[3][1] - dy.astype(np.float64).sum(0)) <= colsum_bound(dy.astype(np.float64)))
    _gemm_check("dH2", tr["dH2"], dYb, bf(W3).T)
    for l in (2, 1, 0):
        Z = tr["Z%d" % l].astype(np.float64)
        sg = 1.0 / (1.0 + np.exp(-Z))
        dZ = tr["dH%d" % l].astype(np.float64) * sg * (1.0 + Z * (1.0 - sg))
        scale = np.abs(tr["dH%d" % l]) * (sg + np.abs(Z) * sg * (1 - sg))
        assert np.all(np.abs(tr["dZ%d" % l] - dZ) <= 2e-6 * scale + 1e-45), ("dZ%d" % l)
        np.testing.assert_array_equal(tr["dZb%d" % l], bf(tr["dZ%d" % l]))
        Hl = tr["X"] if l == 0 else tr["H%d" % (l - 1)]
        _gemm_check("gW%d" % l, gw[l][0], tr["dZb%d" % l].T, Hl.T, rel=1e-4)
        dz = tr["dZ%d" % l].astype(np.float64)
        assert np.all(np.abs(gw[l][1] - dz.sum(0)) <= colsum_bound(dz)), ("gb%d" % l)
        if l > 0:
            _gemm_check("dH%d" % (l - 1), tr["dH%d" % (l - 1)], tr["dZb%d" % l], bf(layers[l][0]).T)
    # end to end against the reference network (its own bf16 rounding points): a bf16 flip of one
    # hidden activation moves the outputs by ~2^-8 of one of 256 terms, hence the norm-wise bars
    yr, gr = mlp_ref.forward_backward(s.weights(), x, dy)
    assert np.linalg.norm(y - yr) / np.linalg.norm(yr) < 1e-3
    o = 0
    for i, n in zip(mlp_ref.DIMS[:-1], mlp_ref.DIMS[1:]):
        for size in (i * n, n):
            a, b = g[o:o + size], gr[o:o + size]
            o += size
            assert np.linalg.norm(a - b) / np.linalg.norm(b) < 5e-3


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_node_spline_path_matches_oracle(oracle_mod, Lb, prec):
    """With the plain generator's own node values (no network), the node-spline log-likelihood
    agrees with the oracle to the spline's accuracy, in FP64 and in mixed precision (where the
    spline phase's sine and cosine are FP32, ~1 ulp of 1, as the FP32 transfer functions)."""
    import torch
    flag = Lb.PE_PREC_MIXED if prec == "mixed" else 0
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
    ll, used = s.loglike([gd], torch.tensor(th, device="cuda"), W.MODE_ALL | flag)
    ll = ll.cpu().numpy()
    assert np.all(used.cpu().numpy() == 1)
    ref, dhhh = oracle_mod.loglike_batch([od], th, W.MODE_ALL)
    dd = od_dd = oracle_mod.loglike([od], inj, 0)["dd"].sum()
    for i in range(th.shape[0]):
        scale = 0.5 * dd + abs(dhhh[i, :, :, 0].sum()) + 0.5 * dhhh[i, :, :, 1].sum()
        H.record_margin("surrogate:node_spline_%s" % prec, abs(ll[i] - ref[i]) / (1e-6 * scale))
        assert abs(ll[i] - ref[i]) <= 1e-6 * scale, (i, ll[i], ref[i])
    s.close()


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_node_spline_path_network_matches_oracle(oracle_mod, Lb, prec):
    """The node-spline path on a two-detector network, LISA (heliocentric) and TianQin (geocentric
    orbit, the FP32 node geometry's other branch), with the plain generator's node values: joint
    log L within the spline's 1e-6 of the likelihood's scale of the oracle's."""
    import torch
    flag = Lb.PE_PREC_MIXED if prec == "mixed" else 0
    T = 2.0 ** 20
    k0, nb = W.grid(T)
    inj = np.array([2e6, 3.0, 0.5, 0.3, 25.8, 0.4, 1.3, 1.375, -1.2108, 2.659, 0.8 * T])
    ods = [H.oracle_detector(oracle_mod, det, T, k0, nb, inj, W.MODE_ALL, seed)
           for det, seed in ((W.LISA, 5), (W.TIANQIN, 6))]
    gds = [H.library_detector(Lb, od) for od in ods]
    s = Lb.Surrogate(seed=1)
    s.set_node_source(1)
    th = np.vstack([inj, W.draw_prior(5, 37, T)])
    th[1:, 0] = np.linspace(4e5, 8e6, 5)
    th[1:, 1] = np.minimum(th[1:, 1], 8.0)
    ll, used = s.loglike(gds, torch.tensor(th, device="cuda"), W.MODE_ALL | flag)
    ll = ll.cpu().numpy()
    assert np.all(used.cpu().numpy() == 1)
    ref, dhhh = oracle_mod.loglike_batch(ods, th, W.MODE_ALL)
    dd = sum(oracle_mod.loglike([od], inj, 0)["dd"].sum() for od in ods)
    for i in range(th.shape[0]):
        scale = 0.5 * dd + abs(dhhh[i, :, :, 0].sum()) + 0.5 * dhhh[i, :, :, 1].sum()
        H.record_margin("surrogate:node_spline_network_%s" % prec, abs(ll[i] - ref[i]) / (1e-6 * scale))
        assert abs(ll[i] - ref[i]) <= 1e-6 * scale, (i, ll[i], ref[i])
    s.close()


def test_heldout_mismatch_acceptance(Lb, lisa22, trained):
    """>= 99% of held-out samples inside the training box have mismatch <= 1e-3 against the plain
    generator on the 2^22 s LISA grid (noise-weighted inner product)."""
    import torch
    th = W.draw_prior(2048, 2606, T22)
    mm = trained.mismatch(lisa22, torch.tensor(th, device="cuda"), W.MODE_ALL).cpu().numpy()
    inbox = (th[:, 0] >= BOX_MLO) & (th[:, 1] <= BOX_QMAX)
    assert inbox.mean() > 0.7
    assert np.all(mm[~inbox] == 0.0)                 # fallback samples are the plain signal
    frac = np.mean(mm[inbox] <= 1e-3)
    assert frac >= 0.99, (frac, np.quantile(mm[inbox], [0.5, 0.99]))


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_fallback_is_the_plain_path_bitwise(Lb, lisa22, trained, prec):
    """Out-of-box samples give the plain path's log L bit for bit, in each precision (the same
    unit, the same per-tile partials and the same fixed-order reduction)."""
    import torch
    flag = Lb.PE_PREC_MIXED if prec == "mixed" else 0
    th = W.draw_prior(64, 2607, T22)
    th[::2, 1] = 10.5                                  # outside the box (q > 10)
    th[1::4, 2] = 0.995                                # outside the box (|chi_1| > 0.99)
    tt = torch.tensor(th, device="cuda")
    ll, used = trained.loglike([lisa22], tt, W.MODE_ALL | flag)
    ref = Lb.loglike([lisa22], th, W.MODE_ALL | flag)["logl"]
    out = (th[:, 1] > BOX_QMAX) | (np.abs(th[:, 2]) > 0.99)
    assert np.array_equal(used.cpu().numpy(), (~out).astype(np.int32))
    assert np.array_equal(ll.cpu().numpy()[out], ref[out])


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_exact_node_values_above_the_network_bound(Lb, lisa22, trained, prec):
    """In-box samples above the network's mass-ratio bound (q > 8) take the plain generator's own
    node values on the spline path: their log L equals the no-network path's bit for bit, while
    the samples below the bound differ from it (network node values)."""
    import torch
    flag = Lb.PE_PREC_MIXED if prec == "mixed" else 0
    th = W.draw_prior(64, 2612, T22)
    th[::2, 1] = np.linspace(8.2, 9.9, 32)             # above the network's bound
    th[1::2, 1] = np.minimum(th[1::2, 1], 7.5)         # below it
    tt = torch.tensor(th, device="cuda")
    ll, used = trained.loglike([lisa22], tt, W.MODE_ALL | flag)
    trained.set_node_source(1)
    try:
        ll_exact, _ = trained.loglike([lisa22], tt, W.MODE_ALL | flag)
    finally:
        trained.set_node_source(0)
    ll, ll_exact = ll.cpu().numpy(), ll_exact.cpu().numpy()
    assert np.all(used.cpu().numpy() == 1)
    assert np.array_equal(ll[::2], ll_exact[::2])
    assert np.all(ll[1::2] != ll_exact[1::2])


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_geocentric_detector_takes_the_plain_path(Lb, trained, prec):
    """A detector on a geocentric orbit (TianQin) never takes the node splines: in-box samples get
    the plain path's log L bit for bit and used = 0."""
    import torch
    flag = Lb.PE_PREC_MIXED if prec == "mixed" else 0
    T = 2.0 ** 20
    k0, nb = W.grid(T)
    d = Lb.Detector(W.TIANQIN, T, k0, nb)
    d.inject(W.theta_injection(T), W.MODE_ALL, W.normals(nb, 11))
    th = W.draw_prior(32, 2611, T)
    th[:, 1] = np.minimum(th[:, 1], 8.0)
    th[:, 0] = np.maximum(th[:, 0], 3e5)
    ll, used = trained.loglike([d], torch.tensor(th, device="cuda"), W.MODE_ALL | flag)
    ref = Lb.loglike([d], th, W.MODE_ALL | flag)["logl"]
    assert np.all(used.cpu().numpy() == 0)
    assert np.array_equal(ll.cpu().numpy(), ref)
    d.close()


def test_precision_flags_that_the_surrogate_rejects(Lb, lisa22, trained):
    """The mismatch study is FP64 only, and the all-FP32 option is not a surrogate path."""
    import torch
    tt = torch.tensor(W.draw_prior(4, 2610, T22), device="cuda")
    for call in (lambda: trained.mismatch(lisa22, tt, W.MODE_ALL | Lb.PE_PREC_MIXED),
                 lambda: trained.loglike([lisa22], tt, W.MODE_ALL | Lb.PE_PREC_FP32),
                 lambda: trained.loglike([lisa22], tt, Lb.PE_PREC_MIXED)):
        with pytest.raises(Lb.PeError) as e:
            call()
        assert e.value.status == Lb.PE_EINVAL


def test_network_against_the_paths_without_it(Lb, lisa22, trained):
    """What the trained network buys, on one in-box batch (1024 samples, 5 modes, 2^22 s LISA),
    device-timed (median of five), at each path's accuracy:
      network     MLP node values (3PN/3.5PN phase terms, |H_lm|) -> node splines -> response;
      no network  the same node splines from the plain generator's exact node values;
      plain FP64  the per-bin path (1e-10 parity);
      plain mixed the per-bin path with double-word geometry (1e-10 parity);
      network mixed / no network mixed: the spline path with PE_PREC_MIXED.
    The spline path beats the plain FP64 path (> 1.3x) with or without the network. In FP64 the
    network buys little over exact node values (TaylorF2 is analytic, so its FP64 node values cost
    about what the MLP inference does); in the mixed path, where the per-bin work has left the FP64
    pipe, the exact node values' FP64 evaluation is a visible share and the BF16 network beats it
    (> 1.15x; measured ~1.4x). The mixed spline path stays within 1e-6 of the likelihood's scale
    of the FP64 spline path and beats the plain mixed path at full parity (> 2x; measured ~4x)."""
    import torch
    th = W.draw_prior(1024, 2608, T22)
    th[:, 1] = np.minimum(th[:, 1], 8.0)
    th[:, 0] = np.maximum(th[:, 0], 3e5)
    tt = torch.tensor(th, device="cuda")
    out = torch.empty(1024, dtype=torch.float64, device="cuda")
    st = torch.cuda.current_stream()

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

    t_plain = med(lambda: Lb.pe_loglike_batch([lisa22.handle], tt, 1024, W.MODE_ALL, out, None, None, st))
    t_mixed = med(lambda: Lb.pe_loglike_batch([lisa22.handle], tt, 1024, W.MODE_ALL | Lb.PE_PREC_MIXED, out, None,
                                              None, st))
    t_net = med(lambda: trained.loglike([lisa22], tt, W.MODE_ALL))
    mm_net = trained.mismatch(lisa22, tt, W.MODE_ALL).cpu().numpy()
    trained.set_node_source(1)
    try:
        t_exact = med(lambda: trained.loglike([lisa22], tt, W.MODE_ALL))
        mm_exact = trained.mismatch(lisa22, tt, W.MODE_ALL).cpu().numpy()
    finally:
        trained.set_node_source(0)
    mx = W.MODE_ALL | Lb.PE_PREC_MIXED
    t_net_mx = med(lambda: trained.loglike([lisa22], tt, mx))
    trained.set_node_source(1)
    try:
        t_exact_mx = med(lambda: trained.loglike([lisa22], tt, mx))
    finally:
        trained.set_node_source(0)
    ll64 = trained.loglike([lisa22], tt, W.MODE_ALL)[0].cpu().numpy()
    llmx = trained.loglike([lisa22], tt, mx)[0].cpu().numpy()
    dh = Lb.loglike([lisa22], tt, W.MODE_ALL, dhhh=True)["dhhh"].cpu().numpy()
    scale = 0.5 * lisa22.data_norm().sum() + np.abs(dh[..., 0].sum(axis=(1, 2))) + 0.5 * dh[..., 1].sum(axis=(1, 2))
    dev = np.max(np.abs(llmx - ll64) / scale)
    print("plain %.2f ms, mixed %.2f ms, network %.2f ms, no network %.2f ms, network mixed %.2f ms, "
          "no network mixed %.2f ms, mixed vs fp64 spline path %.2e of the scale"
          % (t_plain, t_mixed, t_net, t_exact, t_net_mx, t_exact_mx, dev))
    H.record_margin("surrogate:network_over_no_network_speed", t_exact / t_net)
    H.record_margin("surrogate:network_over_plain_fp64_speed", t_plain / t_net)
    H.record_margin("surrogate:network_over_plain_mixed_speed", t_mixed / t_net)
    H.record_margin("surrogate:network_mixed_over_plain_mixed_speed", t_mixed / t_net_mx)
    H.record_margin("surrogate:network_mixed_over_network_fp64_speed", t_net / t_net_mx)
    H.record_margin("surrogate:no_network_mixed_over_plain_mixed_speed", t_mixed / t_exact_mx)
    H.record_margin("surrogate:mixed_vs_fp64_spline_dev_over_1e-6", dev / 1e-6)
    assert np.mean(mm_net <= 1e-3) >= 0.99
    assert np.max(mm_exact) <= 1e-5
    assert t_plain / t_net > 1.3 and t_plain / t_exact > 1.3
    assert dev <= 1e-6
    assert t_net_mx < t_net
    assert t_mixed / t_net_mx > 2.0
    assert t_exact_mx / t_net_mx > 1.15


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
