"""Pins of the surrogate's CPU reference network (oracle/mlp_ref.py), which the GPU tests use for
the tensor-core MLP: its bfloat16 rounding against PyTorch's round-to-nearest-even conversion,
and its hand-written backward pass against central differences of its own forward pass (with the
bf16 rounding points switched off and the layers made small, so that every weight is checked)."""
import numpy as np
import pytest

from oracle import mlp_ref


def test_bf16_rounding_is_round_to_nearest_even():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(11)
    x = np.concatenate([rng.standard_normal(4096) * 10.0 ** rng.integers(-30, 30, 4096),
                        # exact ties between two bf16 neighbours: 1 + k 2^-8 + 2^-9 (even and odd k)
                        1.0 + np.arange(16) * 2.0 ** -8 + 2.0 ** -9,
                        -(1.0 + np.arange(16) * 2.0 ** -8 + 2.0 ** -9)]).astype(np.float32)
    want = torch.from_numpy(x).to(torch.bfloat16).to(torch.float64).numpy()
    np.testing.assert_array_equal(mlp_ref.bf16(x), want)


def test_backward_matches_central_differences(monkeypatch):
    dims = (3, 5, 4, 6, 2)
    monkeypatch.setattr(mlp_ref, "DIMS", dims)
    monkeypatch.setattr(mlp_ref, "bf16", lambda a: np.asarray(a, dtype=np.float64))
    rng = np.random.default_rng(5)
    n = sum(i * o + o for i, o in zip(dims[:-1], dims[1:]))
    w = rng.standard_normal(n) * 0.7
    x = rng.standard_normal((7, dims[0]))
    dy = rng.standard_normal((7, dims[-1]))
    _, g = mlp_ref.forward_backward(w, x, dy)

    def loss(wv):
        y, _ = mlp_ref.forward_backward(wv, x, dy)
        return float((y * dy).sum())

    h = 5e-3
    fd = np.empty(n)
    for i in range(n):
        e = np.zeros(n)
        e[i] = h
        fd[i] = (loss(w + e) - loss(w - e)) / (2 * h)
    # the forward rounds pre-activations to float32 (~6e-8), so differences carry ~1e-5 noise
    assert np.abs(g - fd).max() <= 1e-3 * max(1.0, np.abs(fd).max()), np.abs(g - fd).max()
