"""FP64 reference of the edge-proposal network (test infrastructure only).

y = w3 . relu(W2 relu(W1 x + b1) + b2) + b3 and the gradient of
L = inv_n/2 sum_r mask_r (y_r - t_r)^2.  The network is this project's
stand-in for the edge importance of Sec. 5.3.1; it has no formula in the
thesis.  With ``bf16=True`` the inputs, weights and the intermediate tensors
that the tensor-core kernels store in BF16 (h1, dz2, dz1) are rounded to
BF16 at the same points; all arithmetic is FP64.
"""
import numpy as np


def to_bf16(a):
    """Round float values to the nearest BF16 (ties to even), returned as float64."""
    x = np.ascontiguousarray(a, np.float32)
    u = x.view(np.uint32).astype(np.uint64)
    u = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def bf16_bits(a):
    """BF16 bit patterns (uint16) of float values, round to nearest even."""
    x = np.ascontiguousarray(a, np.float32)
    u = x.view(np.uint32).astype(np.uint64)
    return (((u + 0x7FFF + ((u >> 16) & 1)) >> 16) & 0xFFFF).astype(np.uint16)


def forward(x, p, bf16=True):
    r = to_bf16 if bf16 else (lambda v: np.asarray(v, np.float64))
    X, W1, W2 = r(x), r(p["w1"]), r(p["w2"])
    z1 = X @ W1.T + p["b1"]
    h1 = r(np.maximum(z1, 0.0))
    z2 = h1 @ W2.T + p["b2"]
    h2 = np.maximum(z2, 0.0)
    y = h2 @ np.asarray(p["w3"], np.float64) + float(p["b3"][0])
    return y, dict(X=X, W1=W1, W2=W2, z1=z1, h1=h1, z2=z2, h2=h2)


def backward(x, target, mask, inv_n, p, bf16=True):
    r = to_bf16 if bf16 else (lambda v: np.asarray(v, np.float64))
    y, c = forward(x, p, bf16)
    e = y - target
    loss = 0.5 * inv_n * float(np.sum(mask * e * e))
    dy = mask * e * inv_n
    w3 = np.asarray(p["w3"], np.float64)
    g = {"w3": c["h2"].T @ dy, "b3": np.array([dy.sum()])}
    dz2 = np.where(c["z2"] > 0, dy[:, None] * w3[None, :], 0.0)
    g["b2"] = dz2.sum(0)
    dz2r = r(dz2)
    g["w2"] = dz2r.T @ c["h1"]
    dh1 = dz2r @ c["W2"]
    dz1 = np.where(c["z1"] > 0, dh1, 0.0)
    g["b1"] = dz1.sum(0)
    g["w1"] = r(dz1).T @ c["X"]
    return g, loss


def init_params(seed, n_in=32, hidden=64):
    """He-style initialisation (seeded)."""
    rng = np.random.default_rng(seed)
    return {"w1": rng.normal(0, np.sqrt(2.0 / n_in), (hidden, n_in)).astype(np.float32),
            "b1": np.zeros(hidden, np.float32),
            "w2": rng.normal(0, np.sqrt(2.0 / hidden), (hidden, hidden)).astype(np.float32),
            "b2": np.zeros(hidden, np.float32),
            "w3": rng.normal(0, np.sqrt(1.0 / hidden), hidden).astype(np.float32),
            "b3": np.zeros(1, np.float32)}
