"""Tensor-core network kernels against the FP64 reference (oracle/mlp.py).

The reference rounds inputs, weights and the tensors the kernels store in
BF16 (h1, dz2, dz1) at the same points; remaining differences are FP32
accumulation order and rare one-ulp BF16 rounding flips of an FP32 vs FP64
pre-activation, bounded by 4e-3 of the magnitude of the summed terms.
"""
import numpy as np
import pytest

from oracle import mlp

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1904_12228_gb300 import drt
    return drt, drt.Context(0)


def _device_params(drt, p):
    dev = torch.device("cuda")
    t = {k: torch.from_numpy(np.ascontiguousarray(v, np.float32)).to(dev) for k, v in p.items()}
    t["w1b"] = torch.from_numpy(mlp.bf16_bits(p["w1"]).view(np.int16)).to(dev)
    t["w2b"] = torch.from_numpy(mlp.bf16_bits(p["w2"]).view(np.int16)).to(dev)
    w = drt.MlpWeights(t["w1b"].data_ptr(), t["b1"].data_ptr(), t["w2b"].data_ptr(), t["b2"].data_ptr(),
                       t["w3"].data_ptr(), t["b3"].data_ptr())
    return t, w


def _problem(m, seed):
    rng = np.random.default_rng(seed)
    p = mlp.init_params(seed)
    p["b1"] = rng.normal(0, 0.2, 64).astype(np.float32)
    p["b2"] = rng.normal(0, 0.2, 64).astype(np.float32)
    p["b3"] = np.array([0.3], np.float32)
    x = rng.normal(size=(m, 32)).astype(np.float32)
    return p, x


@pytest.mark.parametrize("m", [1, 127, 1000, 4096])
def test_forward_matches_reference(env, m):
    drt, ctx = env
    p, x = _problem(m, m)
    t, w = _device_params(drt, p)
    xb = torch.from_numpy(mlp.bf16_bits(x).view(np.int16)).cuda()
    y = torch.zeros(m, device="cuda")
    ctx.mlp_forward(xb, w, y)
    torch.cuda.synchronize()
    assert ctx.check_device() == (0, 0)
    want, c = mlp.forward(x, p)
    scale = np.abs(c["h2"]) @ np.abs(p["w3"].astype(np.float64)) + abs(p["b3"][0])
    err = np.abs(y.cpu().numpy() - want)
    assert np.all(err <= 4e-3 * scale + 1e-5), (err.max(), np.argmax(err / (scale + 1e-9)))


@pytest.mark.parametrize("m", [300, 2000])
def test_backward_matches_reference(env, m):
    drt, ctx = env
    p, x = _problem(m, 7 + m)
    rng = np.random.default_rng(m)
    target = rng.normal(size=m).astype(np.float32)
    mask = (rng.uniform(size=m) > 0.3).astype(np.float32)
    inv_n = 1.0 / mask.sum()
    t, w = _device_params(drt, p)
    xb = torch.from_numpy(mlp.bf16_bits(x).view(np.int16)).cuda()
    g = {k: torch.zeros(v.shape, device="cuda") for k, v in p.items()}
    gp = drt.MlpGrads(*(g[k].data_ptr() for k in ("w1", "b1", "w2", "b2", "w3", "b3")))
    loss = torch.zeros(1, device="cuda")
    ctx.mlp_backward(xb, torch.from_numpy(target).cuda(), torch.from_numpy(mask).cuda(), inv_n, w, gp, loss)
    torch.cuda.synchronize()
    assert ctx.check_device() == (0, 0)
    want, wl = mlp.backward(x, target, mask, inv_n, p)
    # magnitude of the summed terms, per gradient entry
    abs_p = {k: np.abs(v.astype(np.float64)) for k, v in p.items()}
    _, cabs = mlp.forward(np.abs(x), abs_p)
    for k in ("w1", "b1", "w2", "b2", "w3", "b3"):
        got = g[k].cpu().numpy().astype(np.float64)
        ref = want[k]
        tol = 4e-3 * np.abs(ref).max() + 1e-6
        assert np.all(np.abs(got - ref) <= tol), (k, np.abs(got - ref).max(), tol)
    assert abs(loss.item() - wl) <= 4e-3 * wl + 1e-6


def test_adam_step_matches_textbook(env):
    drt, ctx = env
    rng = np.random.default_rng(1)
    n = 5000
    p = rng.normal(size=n).astype(np.float32)
    gr = rng.normal(size=n).astype(np.float32)
    pt, gt = torch.from_numpy(p.copy()).cuda(), torch.from_numpy(gr).cuda()
    m1, m2 = torch.zeros(n, device="cuda"), torch.zeros(n, device="cuda")
    pb = torch.zeros(n, dtype=torch.int16, device="cuda")
    mm, vv, pp = np.zeros(n), np.zeros(n), p.astype(np.float64)
    for step in (1, 2, 3):
        ctx.adam_step(pt, gt, m1, m2, pb, lr=1e-2, step=step)
        mm = 0.9 * mm + 0.1 * gr
        vv = 0.999 * vv + 0.001 * gr.astype(np.float64) ** 2
        pp = pp - 1e-2 * (mm / (1 - 0.9 ** step)) / (np.sqrt(vv / (1 - 0.999 ** step)) + 1e-8)
    torch.cuda.synchronize()
    assert np.allclose(pt.cpu().numpy(), pp, rtol=1e-5, atol=1e-6)
    assert np.array_equal(pb.cpu().numpy().view(np.uint16), mlp.bf16_bits(pt.cpu().numpy()))


def test_training_fits_a_smooth_function(env):
    drt, ctx = env
    rng = np.random.default_rng(3)
    m = 4096
    x = rng.uniform(-1, 1, size=(m, 32)).astype(np.float32)
    target = (np.sin(2 * x[:, 0]) + x[:, 1] * x[:, 2] + 0.5 * np.abs(x[:, 3])).astype(np.float32)
    p = mlp.init_params(5)
    t, w = _device_params(drt, p)
    xb = torch.from_numpy(mlp.bf16_bits(x).view(np.int16)).cuda()
    tg, mk = torch.from_numpy(target).cuda(), torch.ones(m, device="cuda")
    names = ("w1", "b1", "w2", "b2", "w3", "b3")
    g = {k: torch.zeros_like(t[k]) for k in names}
    st = {k: (torch.zeros_like(t[k]), torch.zeros_like(t[k])) for k in names}
    gp = drt.MlpGrads(*(g[k].data_ptr() for k in names))
    losses = []
    for step in range(1, 301):
        for k in names:
            g[k].zero_()
        loss = torch.zeros(1, device="cuda")
        ctx.mlp_backward(xb, tg, mk, 1.0 / m, w, gp, loss)
        for k in names:
            ctx.adam_step(t[k], g[k], st[k][0], st[k][1], t.get(k + "b"), lr=3e-3, step=step)
        losses.append(loss.item())
    assert losses[-1] < 0.1 * losses[0], (losses[0], losses[-1])
