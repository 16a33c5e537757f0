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


def _train_problem(rng, rows_per_log=(700, 1300)):
    logs = []
    for n in rows_per_log:
        x = rng.normal(size=(n, 32)).astype(np.float32)
        seg_log = (rng.exponential(size=n) * (rng.uniform(size=n) > 0.2)).astype(np.float32)
        seg_len = rng.uniform(0.1, 30.0, size=n)
        logs.append((x, seg_log, seg_len, float(16 * 96 * 96)))
    return logs


def _reference_rows(logs, seed, delta=1e-3):
    """Targets, weights and shuffle of drt_mlp_train, written out in numpy."""
    import oracle
    tgt, msk, xs = [], [], []
    for x, seg_log, seg_len, N in logs:
        S, L = float(np.sum(seg_log.astype(np.float64))), float(np.sum(seg_len))
        dens = seg_log.astype(np.float64) * (L / N) / np.maximum(seg_len, 1e-12)
        tgt.append(np.log(dens / max(S / N, 1e-30) + delta))
        msk.append(seg_len / (L / len(seg_len)))
        xs.append(x)
    tgt, msk, xs = np.concatenate(tgt), np.concatenate(msk), np.concatenate(xs)
    key = np.array([seed & 0xFFFFFFFF, seed >> 32], np.uint32)
    keys = np.array([oracle.philox(np.array([r, 0, 0x4D4C5054, 0], np.uint32), key)[0] for r in range(len(tgt))],
                    np.uint64)
    perm = np.argsort(keys, kind="stable")
    return tgt[perm], msk[perm], xs[perm], perm


def _device_logs(drt, logs):
    held, recs = [], []
    for x, seg_log, seg_len, N in logs:
        t = (torch.from_numpy(mlp.bf16_bits(x).view(np.int16)).cuda(), torch.from_numpy(seg_log).cuda(),
             torch.from_numpy(seg_len).cuda())
        held.append(t)
        recs.append(drt.MlpLog(t[0].data_ptr(), t[1].data_ptr(), t[2].data_ptr(), len(seg_log), N))
    return held, recs


def _state(drt, p):
    names = ("w1", "b1", "w2", "b2", "w3", "b3")
    t, _ = _device_params(drt, p)
    m1 = {k: torch.zeros_like(t[k]) for k in names}
    m2 = {k: torch.zeros_like(t[k]) for k in names}
    g = {k: torch.zeros_like(t[k]) for k in names}
    st = drt.MlpState()
    for i, k in enumerate(names):
        st.p[i], st.m1[i], st.m2[i], st.g[i] = t[k].data_ptr(), m1[k].data_ptr(), m2[k].data_ptr(), g[k].data_ptr()
    st.w1_bf16, st.w2_bf16, st.step = t["w1b"].data_ptr(), t["w2b"].data_ptr(), 0
    return st, t, m1, m2, g


def test_mlp_train_prepares_the_rows_as_specified(env):
    """drt_mlp_train's targets, regression weights and shuffle against their
    definition, written out in numpy (targets in FP32 of an FP64 value)."""
    drt, ctx = env
    rng = np.random.default_rng(11)
    logs = _train_problem(rng)
    held, recs = _device_logs(drt, logs)
    st, *_ = _state(drt, mlp.init_params(3))
    rows = sum(len(l[1]) for l in logs)
    tg = torch.zeros(rows, device="cuda")
    mk = torch.zeros(rows, device="cuda")
    ix = torch.zeros(rows, dtype=torch.int64, device="cuda")
    seed = (7 << 32) + 12345
    ctx.mlp_train(recs, st, 0, seed=seed, rows_target=tg, rows_mask=mk, rows_index=ix)
    want_t, want_m, _, perm = _reference_rows(logs, seed)
    assert np.array_equal(ix.cpu().numpy(), perm)
    assert np.allclose(tg.cpu().numpy(), want_t, rtol=1e-6, atol=1e-6)
    assert np.allclose(mk.cpu().numpy(), want_m, rtol=1e-6, atol=0)
    assert st.step == 0


def test_mlp_train_step_matches_the_reference(env):
    """One training step: the gradient on the first shuffled batch against
    the FP64 reference, and the weights after it against bias-corrected Adam
    applied to that gradient at the step's learning rate."""
    drt, ctx = env
    rng = np.random.default_rng(12)
    logs = _train_problem(rng)
    held, recs = _device_logs(drt, logs)
    p = mlp.init_params(4)
    st, t, m1, m2, g = _state(drt, p)
    seed, batch, lr = 99, 512, 2e-3
    loss = torch.zeros(1, device="cuda")
    ctx.mlp_train(recs, st, 1, batch=batch, lr=lr, seed=seed, loss=loss)
    torch.cuda.synchronize()
    assert ctx.check_device() == (0, 0)
    assert st.step == 1
    want_t, want_m, xs, _ = _reference_rows(logs, seed)
    want_g, want_loss = mlp.backward(xs[:batch], want_t[:batch], want_m[:batch], 1.0 / batch, p)
    for k in ("w1", "b1", "w2", "b2", "w3", "b3"):
        got = g[k].cpu().numpy().astype(np.float64)
        assert np.all(np.abs(got - want_g[k]) <= 4e-3 * np.abs(want_g[k]).max() + 1e-6), k
        # Adam's first step from zero moments, on the gradient the library used
        gk = got.astype(np.float32).astype(np.float64)
        m = 0.1 * gk
        v = 0.001 * gk * gk
        upd = lr * (m / 0.1) / (np.sqrt(v / 0.001) + 1e-8)  # schedule factor at step 0 is 1
        want_p = np.asarray(p[k], np.float64) - upd
        assert np.allclose(t[k].cpu().numpy(), want_p, rtol=1e-5, atol=1e-6), k
    assert abs(loss.item() - want_loss) <= 4e-3 * want_loss + 1e-6
    assert np.array_equal(t["w1b"].cpu().numpy().view(np.uint16), mlp.bf16_bits(t["w1"].cpu().numpy()))


def test_mlp_train_options_are_checked(env):
    drt, ctx = env
    rng = np.random.default_rng(13)
    logs = _train_problem(rng, (50,))
    x, seg_log, seg_len, N = logs[0]
    st, *_ = _state(drt, mlp.init_params(5))
    bad = [drt.MlpLog(torch.zeros(1).data_ptr(), 0, 0, 50, N)]  # host / NULL arrays
    with pytest.raises(drt.DrtError):
        ctx.mlp_train(bad, st, 1)
    held, recs = _device_logs(drt, logs)
    recs[0].n_samples = 0.0
    with pytest.raises(drt.DrtError):
        ctx.mlp_train(recs, st, 1)
