"""Pin of the FP64 network reference: its analytic gradient equals central
finite differences of its own forward pass (no BF16 rounding), and the BF16
rounding helper rounds to nearest even."""
import numpy as np

from oracle import mlp


def test_bf16_rounding():
    vals = np.array([1.0, 1.0 + 2 ** -8, 1.0 + 3 * 2 ** -9, -2.5, 3.14159265], np.float32)
    r = mlp.to_bf16(vals)
    assert r[0] == 1.0 and r[1] == 1.0 and r[2] == 1.0 + 2 ** -7 and r[3] == -2.5
    assert abs(r[4] - 3.140625) < 1e-12


def test_gradient_matches_finite_differences():
    rng = np.random.default_rng(0)
    p = {k: v.astype(np.float64) for k, v in mlp.init_params(3).items()}
    p["b1"] = rng.normal(0, 0.1, 64)
    p["b2"] = rng.normal(0, 0.1, 64)
    x = rng.normal(size=(50, 32))
    t = rng.normal(size=50)
    mask = (rng.uniform(size=50) > 0.2).astype(np.float64)
    g, loss = mlp.backward(x, t, mask, 1.0 / mask.sum(), p, bf16=False)
    h = 1e-6
    for name in ("w1", "b1", "w2", "b2", "w3", "b3"):
        flat = p[name].reshape(-1)
        for idx in rng.choice(len(flat), size=min(6, len(flat)), replace=False):
            old = flat[idx]
            flat[idx] = old + h
            lp = mlp.backward(x, t, mask, 1.0 / mask.sum(), p, bf16=False)[1]
            flat[idx] = old - h
            lm = mlp.backward(x, t, mask, 1.0 / mask.sum(), p, bf16=False)[1]
            flat[idx] = old
            fd = (lp - lm) / (2 * h)
            assert abs(fd - g[name].reshape(-1)[idx]) < 1e-6 * max(1.0, abs(fd)), (name, idx)
