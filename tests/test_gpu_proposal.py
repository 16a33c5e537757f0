"""The learned primary-edge proposal: trained on the GPU by the network
kernels from logs of the plain sampler, it must keep the gradient unbiased
and lower gradient variance x time on scenes it did not see."""
import numpy as np
import pytest

from paper_1904_12228_gb300 import scenegen as sg

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def trained():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1904_12228_gb300 import drt, proposal as P
    ctx = drt.Context(0)
    parts = []
    for seed in range(100, 108):
        sc = sg.direct_lighting(seed, width=96, height=96, subdiv=3)
        s = drt.Scene.from_arrays(ctx, sc)
        w = torch.from_numpy(sg.loss_adjoint(seed, sc.width, sc.height)).cuda()
        parts.append(P.collect(ctx, s, w, edge_spp=16, passes=4, seed=seed * 1000))
    for seed in (116, 117):
        sc = sg.procedural(seed, n_target=20000, width=128, height=128)
        s = drt.Scene.from_arrays(ctx, sc)
        w = torch.from_numpy(sg.loss_adjoint(seed, sc.width, sc.height)).cuda()
        parts.append(P.collect(ctx, s, w, edge_spp=8, passes=4, seed=seed * 1000, max_depth=3))
    data = P.Dataset(parts)
    net = P.EdgeProposal(ctx, 0)
    # the library trains: targets, shuffle, schedule and steps (drt_mlp_train)
    hist = [net.fit(data, steps=100, batch=8192, seed=1), net.fit(data, steps=1400, batch=8192, seed=2)]
    return ctx, P, net, hist


def test_training_lowers_the_loss(trained):
    _, _, net, hist = trained
    assert np.all(np.isfinite(hist))
    assert hist[-1] < 0.8 * hist[0], hist
    assert net.steps == 1500


@pytest.mark.parametrize("kind,seed", [("direct", 200), ("procedural", 202)])
def test_learned_proposal_beats_plain_on_held_out_scene(trained, kind, seed):
    ctx, P, net, _ = trained
    from paper_1904_12228_gb300 import drt
    if kind == "direct":
        sc, md, es = sg.direct_lighting(seed, width=96, height=96, subdiv=3), 1, 16
    else:
        sc, md, es = sg.procedural(seed, n_target=20000, width=128, height=128), 3, 8
    s = drt.Scene.from_arrays(ctx, sc)
    w = torch.from_numpy(sg.loss_adjoint(seed, sc.width, sc.height)).cuda()
    plain, learned, ratio, z2 = P.compare(s, w, net, edge_spp=es, K=48, seed=seed * 7, max_depth=md)
    assert ctx.check_device() == (0, 0)
    # both estimators unbiased: the mean gradients agree within their errors
    # (mean squared z-score about 1 for 48 runs each)
    assert z2 < 1.5, z2
    # variance x time below the plain sampler's
    assert learned.var < 0.8 * plain.var, (learned.var, plain.var)
    assert ratio < 0.9, (ratio, learned.ms, plain.ms)


def test_scores_cover_every_segment(trained):
    ctx, P, net, _ = trained
    from paper_1904_12228_gb300 import drt
    sc = sg.direct_lighting(201, width=80, height=56, subdiv=2)
    s = drt.Scene.from_arrays(ctx, sc)
    w = torch.from_numpy(sg.loss_adjoint(201, sc.width, sc.height)).cuda()
    y = net.scores(s, w)
    torch.cuda.synchronize()
    assert y.shape[0] == s.num_segments() == len(s.segments()[0])
    assert torch.isfinite(y).all()
    # the image features are zero without an image and present with one
    x0 = net.features(s, w).view(torch.bfloat16).float()
    x1 = net.features(s, w, image=P.step_image(s, 3)).view(torch.bfloat16).float()
    torch.cuda.synchronize()
    assert torch.isfinite(x1).all()
    assert float(x0[:, 30:32].abs().max()) == 0.0 and float(x1[:, 30:32].abs().max()) > 0.0
    assert torch.equal(x0[:, :30], x1[:, :30])
    assert float(x1[:, 29].min()) >= 0.0 and float(x1[:, 29].max()) > 0.0
