"""The method against central finite differences on the GPU.

The CUDA path matches the oracle sample for sample (test_gpu_parity.py), so
finite differences of the GPU image at very high sample counts check the
method itself -- the readings of the edge terms -- where CPU finite
differences are too noisy: in particular the solid-angle form of the
secondary edge term for reflected light (depth 2), which the blocker of the
GI scene exercises through its indirect shadow on the panel.

Both sides are Monte Carlo estimates: a z-test over seeds (Sec. 5.4.1 uses
central differences with far more samples for the same purpose).
"""
import numpy as np
import pytest

from paper_1904_12228_gb300 import scenegen as sg

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _setup(scene):
    from paper_1904_12228_gb300 import drt
    ctx = drt.Context(0)
    return drt, ctx


def _loss(drt, ctx, scene, verts, w, spp, seed, depth):
    sc = scene.copy()
    sc.verts = verts.astype(np.float32)
    s = drt.Scene.from_arrays(ctx, sc)
    img = torch.zeros((scene.height, scene.width, 3), device="cuda")
    s.render(img, drt.make_opts(spp, 1, max_depth=depth, seed=seed))
    return float((img.double() * w).sum().item())


def _grad(drt, ctx, scene, w, spp, seed, depth):
    s = drt.Scene.from_arrays(ctx, scene)
    img = torch.zeros((scene.height, scene.width, 3), device="cuda")
    opts = drt.make_opts(spp, spp, max_depth=depth, seed=seed)
    tape = s.render(img, opts, want_tape=True)
    dv = torch.zeros((len(scene.verts), 3), device="cuda")
    s.backward(w.float().contiguous(), opts, tape=tape, d_verts=dv)
    torch.cuda.synchronize()
    return dv.double().cpu().numpy()


@pytest.mark.parametrize("name,depth", [("gi_panel", 2), ("direct", 1)])
def test_gradient_matches_central_differences_on_gpu(name, depth):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    if name == "gi_panel":
        scene = sg.gi_panel(16, 16)
        probes = [(12, 0), (12, 2), (13, 1), (14, 0), (5, 1), (6, 0)]
        w = torch.ones((16, 16, 3), dtype=torch.float64, device="cuda")
    else:
        scene = sg.direct_lighting(1236, width=16, height=16, subdiv=1)
        V = len(scene.verts)
        probes = [(0, 0), (0, 1), (V - 8, 1), (V - 3, 0), (V - 2, 2)]
        w = torch.from_numpy(sg.loss_adjoint(4, 16, 16)).double().cuda()
    drt, ctx = _setup(scene)
    K = 8
    ours = np.array([[_grad(drt, ctx, scene, w, 4096, 100 + k, depth)[v, c] for v, c in probes] for k in range(K)])
    h = 1e-2
    fd = []
    for k in range(K):
        row = []
        for v, c in probes:
            vp, vm = scene.verts.astype(np.float64).copy(), scene.verts.astype(np.float64).copy()
            vp[v, c] += h
            vm[v, c] -= h
            row.append((_loss(drt, ctx, scene, vp, w, 65536, 7000 + k, depth) -
                        _loss(drt, ctx, scene, vm, w, 65536, 7000 + k, depth)) / (2 * h))
        fd.append(row)
    fd = np.array(fd)
    se = np.sqrt(ours.var(0, ddof=1) / K + fd.var(0, ddof=1) / K)
    z = np.abs(ours.mean(0) - fd.mean(0)) / se
    assert np.all(z < 4.5), list(zip(probes, ours.mean(0), fd.mean(0), se))
    assert np.abs(ours.mean(0)).max() > 10 * se.max() or name == "direct"
