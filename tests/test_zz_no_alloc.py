"""drt_render_backward_noalloc: the backward pass for callers that cannot
allocate device memory during their step (a loop whose device memory is
reserved up front by its own caching allocator, or a fixed memory budget).

It must give the gradients of drt_render_backward, within the parity
tolerance of the other GPU tests, on consecutive calls that share its fixed
scratch array.  This file is collected last so that a failure here comes
after every other test has run.
"""
import numpy as np
import pytest

import oracle
from paper_1904_12228_gb300 import scenegen as sg

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _flat(*ts):
    return np.concatenate([t.cpu().numpy().ravel().astype(np.float64) for t in ts])


def _zeros(scene):
    V, T = len(scene.verts), len(scene.tris)
    return dict(d_verts=torch.zeros((V, 3), device="cuda"), d_albedo=torch.zeros((T, 3), device="cuda"),
                d_radiance=torch.zeros(3, device="cuda"), d_cam_to_world=torch.zeros((3, 4), device="cuda"),
                d_cam_scale=torch.zeros(1, device="cuda"))


def test_noalloc_backward_matches_backward_on_consecutive_calls():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1904_12228_gb300 import drt
    ctx = drt.Context(0)
    scene = sg.direct_lighting(1236, width=40, height=28, subdiv=2)
    S = drt.Scene.from_arrays(ctx, scene)
    opts = drt.make_opts(8, 8, seed=11)
    img = torch.zeros((28, 40, 3), device="cuda")
    tape = S.render(img, opts, want_tape=True)
    w = torch.from_numpy(sg.loss_adjoint(3, 40, 28)).cuda()
    ref = _zeros(scene)
    S.backward(w, opts, tape=tape, **ref)
    torch.cuda.synchronize()
    want = _flat(*ref.values())
    _, absum = oracle.backward(scene, w.cpu().numpy(), spp=8, edge_spp=8, seed=11)
    for call in range(2):
        got = _zeros(scene)
        S.backward_noalloc(w, opts, tape=tape, **got)
        torch.cuda.synchronize()
        g = _flat(*got.values())
        err = np.abs(g - want)
        bound = 1e-4 * np.abs(want) + 1e-6 * absum + 1e-12
        assert np.all(err <= bound), "call %d: %d entries off" % (call, int((err > bound).sum()))
        assert np.abs(g).max() > 0
    assert ctx.check_device() == (0, 0)


def test_noalloc_backward_allocates_nothing_and_records_into_a_graph():
    """After one warm call the entry point allocates no device memory (free
    memory unchanged around a call) and records into a CUDA graph captured in
    global mode, where an allocation or a synchronising call ends the capture
    with an error; the replayed graph gives the oracle's gradients."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1904_12228_gb300 import drt
    ctx = drt.Context(0)
    scene = sg.direct_lighting(1236, width=40, height=28, subdiv=2)
    S = drt.Scene.from_arrays(ctx, scene)
    opts = drt.make_opts(8, 8, seed=13)
    img = torch.zeros((28, 40, 3), device="cuda")
    tape = S.render(img, opts, want_tape=True)
    w = torch.from_numpy(sg.loss_adjoint(4, 40, 28)).cuda()
    got = _zeros(scene)
    S.backward_noalloc(w, opts, tape=tape, **got)  # warm call
    torch.cuda.synchronize()
    for t in got.values():
        t.zero_()
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    S.backward_noalloc(w, opts, tape=tape, **got)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    for t in got.values():
        t.zero_()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, capture_error_mode="global"):
        S.backward_noalloc(w, opts, tape=tape, **got)
    for t in got.values():
        t.zero_()
    g.replay()
    torch.cuda.synchronize()
    assert ctx.check_device() == (0, 0)
    want, absum = oracle.backward(scene, w.cpu().numpy(), spp=8, edge_spp=8, seed=13)
    gr = _flat(*got.values())
    err = np.abs(gr - want)
    bound = 1e-4 * np.abs(want) + 1e-6 * absum + 1e-12
    assert np.all(err <= bound), "%d entries off" % int((err > bound).sum())
    assert np.abs(gr).max() > 0


def test_noalloc_backward_matches_backward_at_depth_two():
    """The allocation-free backward evaluates the secondary edge samples inside
    the path pass; the regular backward queues and traces them apart."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1904_12228_gb300 import drt
    ctx = drt.Context(0)
    scene = sg.direct_lighting(1237, width=24, height=20, subdiv=1)
    S = drt.Scene.from_arrays(ctx, scene)
    opts = drt.make_opts(6, 6, max_depth=2, seed=5)
    img = torch.zeros((20, 24, 3), device="cuda")
    tape = S.render(img, opts, want_tape=True)
    w = torch.from_numpy(sg.loss_adjoint(4, 24, 20)).cuda()
    ref = _zeros(scene)
    S.backward(w, opts, tape=tape, **ref)
    got = _zeros(scene)
    S.backward_noalloc(w, opts, tape=tape, **got)
    torch.cuda.synchronize()
    want, g = _flat(*ref.values()), _flat(*got.values())
    _, absum = oracle.backward(scene, w.cpu().numpy(), spp=6, edge_spp=6, seed=5, max_depth=2)
    bound = 1e-4 * np.abs(want) + 1e-6 * absum + 1e-12
    assert np.all(np.abs(g - want) <= bound), int((np.abs(g - want) > bound).sum())
    assert np.abs(g).max() > 0
    assert ctx.check_device() == (0, 0)


def test_noalloc_backward_rejects_host_arrays_and_oversize_images():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1904_12228_gb300 import drt
    ctx = drt.Context(0)
    scene = sg.direct_lighting(1236, width=16, height=12, subdiv=1)
    S = drt.Scene.from_arrays(ctx, scene)
    opts = drt.make_opts(4, 4, seed=1)
    host = np.zeros((12, 16, 3), np.float32)
    with pytest.raises(drt.DrtError) as e:
        S.backward_noalloc(host, opts, d_verts=torch.zeros((len(scene.verts), 3), device="cuda"))
    assert e.value.status == 1
    big = sg.direct_lighting(1236, width=1024, height=1024, subdiv=1)
    B = drt.Scene.from_arrays(ctx, big)
    wd = torch.zeros((1024, 1024, 3), device="cuda")
    with pytest.raises(drt.DrtError) as e:
        B.backward_noalloc(wd, drt.make_opts(32, 32, seed=1), d_verts=torch.zeros((len(big.verts), 3), device="cuda"))
    assert e.value.status == 1 and "maximum" in str(e.value)
