"""Reference of the surrogate's dense network (numpy, FP64 accumulation), used by the tests to
check the tensor-core forward and backward kernels. TEST INFRASTRUCTURE ONLY.

It rounds to bfloat16 (round to nearest even) at the points where the tensor-core path stores
bf16 operands: the input features, every weight matrix, every SiLU activation, the output
cotangent and the pre-activation cotangents fed to the weight-gradient and input-gradient
products. Bias gradients use the unrounded fp32 cotangents, as the device does.
Network: Z_l = H_{l-1} W_l^T + b_l, H_l = SiLU(Z_l) for l = 0, 1, 2; Y = H_2 W_3^T + b_3.
"""
import numpy as np

DIMS = (64, 256, 256, 256, 2560)


def bf16(a: np.ndarray) -> np.ndarray:
    a32 = np.ascontiguousarray(a, dtype=np.float32)
    u = a32.view(np.uint32).astype(np.uint64)
    rounded = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return rounded.astype(np.uint32).view(np.float32).astype(np.float64)


def unpack(w: np.ndarray):
    """Split the flat [W0, b0, W1, b1, W2, b2, W3, b3] vector ([out][in] weights)."""
    layers, o = [], 0
    for l in range(4):
        i, n = DIMS[l], DIMS[l + 1]
        W = w[o:o + i * n].reshape(n, i).astype(np.float64)
        o += i * n
        b = w[o:o + n].astype(np.float64)
        o += n
        layers.append((W, b))
    return layers


def silu(z):
    return z / (1.0 + np.exp(-z))


def forward_backward(w_flat: np.ndarray, x: np.ndarray, dy: np.ndarray):
    layers = unpack(w_flat)
    H = bf16(x)
    Hs, Zs = [H], []
    for l in range(3):
        W, b = layers[l]
        Z = (H @ bf16(W).T + b).astype(np.float32).astype(np.float64)
        Zs.append(Z)
        H = bf16(silu(Z))
        Hs.append(H)
    W3, b3 = layers[3]
    Y = H @ bf16(W3).T + b3
    grads = []
    dYb = bf16(dy)
    gW3 = dYb.T @ Hs[3]
    gb3 = dy.astype(np.float64).sum(axis=0)
    dH = dYb @ bf16(W3)
    g = [(gW3, gb3)]
    for l in (2, 1, 0):
        Z = Zs[l]
        s = 1.0 / (1.0 + np.exp(-Z))
        dZ = dH * s * (1.0 + Z * (1.0 - s))
        dZb = bf16(dZ)
        gW = dZb.T @ Hs[l]
        gb = dZ.sum(axis=0)
        g.append((gW, gb))
        if l > 0:
            W, _ = layers[l]
            dH = dZb @ bf16(W)
    g = g[::-1]
    flat = np.concatenate([np.concatenate([gW.ravel(), gb]) for gW, gb in g])
    return Y, flat
