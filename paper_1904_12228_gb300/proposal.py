"""Learned proposal for primary edge samples.

The plain sampler of Sec. 5.2.1 picks a clipped silhouette edge with
probability proportional to its screen length.  Most of those samples land
where the integrand does not jump (hidden edges, edges between faces of equal
colour) and contribute nothing.  Here a 3-layer network (64 wide, BF16 weights
on the tensor cores, FP32 accumulation; drt_mlp_forward) scores each screen
tile segment of every clipped edge; the renderer's proposal 2 draws a segment
with probability q = 1/2 len/L + 1/2 m/M, with m = len * exp(score), and a
point uniformly on it, and divides the sample by its density (Eq. mc with
that pdf).  Half the samples still follow the length distribution, so every
point keeps a nonzero density and the estimator stays unbiased whatever the
network outputs.  This plays the part of the edge importance of Sec. 5.3.1.

Training data comes from the plain sampler itself: a backward pass with the
length distribution over the same segments adds |w (f_u - f_l)| of every
primary edge sample to its segment (seg_log), which estimates the segment's
integral of the edge integrand's magnitude.  The network regresses the log of
that integral per unit length, relative to the scene's mean, weighted by
segment length; drt_mlp_backward and drt_adam_step train it on the GPU.

The figure of merit is gradient variance x time at equal sample count
against the plain sampler, on scenes the network did not see.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np
import torch

from . import drt

NAMES = ("w1", "b1", "w2", "b2", "w3", "b3")
N_IN, HIDDEN = 32, 64
TERM_PRIMARY = 2


def _bf16_bits(t: torch.Tensor) -> torch.Tensor:
    return t.to(torch.bfloat16).view(torch.int16)


class EdgeProposal:
    """Network weights (FP32 masters + BF16 copies), Adam state, gradients."""

    def __init__(self, ctx: drt.Context, seed: int = 0, device: str = "cuda"):
        self.ctx = ctx
        g = torch.Generator().manual_seed(seed)
        shapes = {"w1": (HIDDEN, N_IN), "b1": (HIDDEN,), "w2": (HIDDEN, HIDDEN), "b2": (HIDDEN,), "w3": (HIDDEN,),
                  "b3": (1,)}
        fan_in = {"w1": N_IN, "w2": HIDDEN, "w3": HIDDEN}
        p = {}
        for k, shp in shapes.items():
            if k in fan_in:  # uniform He initialisation for ReLU layers
                lim = math.sqrt(6.0 / fan_in[k]) if k != "w3" else math.sqrt(3.0 / fan_in[k])
                p[k] = (torch.rand(shp, generator=g) * 2 - 1) * lim
            else:
                p[k] = torch.zeros(shp)
        self.p = {k: v.float().to(device).contiguous() for k, v in p.items()}
        self.pb = {k: _bf16_bits(self.p[k]).contiguous() for k in ("w1", "w2")}
        self.g = {k: torch.zeros_like(v) for k, v in self.p.items()}
        self.m1 = {k: torch.zeros_like(v) for k, v in self.p.items()}
        self.m2 = {k: torch.zeros_like(v) for k, v in self.p.items()}
        self.steps = 0
        self._w = drt.MlpWeights(self.pb["w1"].data_ptr(), self.p["b1"].data_ptr(), self.pb["w2"].data_ptr(),
                                 self.p["b2"].data_ptr(), self.p["w3"].data_ptr(), self.p["b3"].data_ptr())
        self._gp = drt.MlpGrads(*(self.g[k].data_ptr() for k in NAMES))

    # -- training resume ------------------------------------------------------
    _MAGIC = b"DRTMLP01"

    def save(self, path: str) -> None:
        """Weights and Adam state as one raw little-endian file: the 8-byte
        tag DRTMLP01, the Adam step count (int64), then for w1 b1 w2 b2 w3 b3
        in turn the FP32 master weights, first moments and second moments
        (row-major, the shapes of the network)."""
        with open(path, "wb") as f:
            f.write(self._MAGIC)
            f.write(np.asarray([self.steps], "<i8").tobytes())
            for k in NAMES:
                for d in (self.p, self.m1, self.m2):
                    f.write(d[k].detach().cpu().numpy().astype("<f4").tobytes())

    def load(self, path: str) -> None:
        """Read a file written by save() into this network, in place (the
        library holds pointers to these arrays), and refresh the BF16 copies
        the forward pass reads."""
        with open(path, "rb") as f:
            raw = f.read()
        if raw[:8] != self._MAGIC:
            raise ValueError("not a network file: bad tag")
        need = 16 + 4 * 3 * sum(self.p[k].numel() for k in NAMES)
        if len(raw) != need:
            raise ValueError("network file of %d bytes, expected %d" % (len(raw), need))
        steps = int(np.frombuffer(raw[8:16], "<i8")[0])
        off = 16
        for k in NAMES:
            for d in (self.p, self.m1, self.m2):
                n = d[k].numel()
                arr = np.frombuffer(raw[off:off + 4 * n], "<f4").astype(np.float32).reshape(tuple(d[k].shape))
                d[k].copy_(torch.from_numpy(arr))
                off += 4 * n
        self.steps = steps
        for k in ("w1", "w2"):
            self.pb[k].copy_(_bf16_bits(self.p[k]))

    # -- inference ------------------------------------------------------------
    def features(self, scene: drt.Scene, d_image: torch.Tensor, n: int | None = None, image=None, stream=None):
        n = scene.num_segments(stream) if n is None else n
        x = torch.empty((n, N_IN), dtype=torch.int16, device=d_image.device)
        if n:
            scene.segment_features(d_image, x, image, stream)
        return x

    def scores(self, scene: drt.Scene, d_image: torch.Tensor, n: int | None = None, image=None, stream=None):
        """Network scores of the scene's current tile segments ([n] float32);
        ``image``: the rendered image of the step (its contrast across edges
        is a feature)."""
        x = self.features(scene, d_image, n, image, stream)
        y = torch.empty(x.shape[0], dtype=torch.float32, device=x.device)
        if x.shape[0]:
            self.ctx.mlp_forward(x, self._w, y, stream)
        return y

    # -- training -------------------------------------------------------------
    def train_step(self, x, target, mask, lr: float, loss: torch.Tensor, stream=None):
        """One Adam step on rows x [m,32] (bf16 bits) with weights mask."""
        for k in NAMES:
            self.g[k].zero_()
        inv_n = 1.0 / max(1, x.shape[0])
        self.ctx.mlp_backward(x, target, mask, inv_n, self._w, self._gp, loss, stream)
        self.steps += 1
        for k in NAMES:
            self.ctx.adam_step(self.p[k], self.g[k], self.m1[k], self.m2[k], self.pb.get(k), lr, self.steps,
                               stream=stream)

    def state(self) -> drt.MlpState:
        """The library's view of the parameters, Adam moments and gradients."""
        st = drt.MlpState()
        for i, k in enumerate(NAMES):
            st.p[i] = self.p[k].data_ptr()
            st.m1[i] = self.m1[k].data_ptr()
            st.m2[i] = self.m2[k].data_ptr()
            st.g[i] = self.g[k].data_ptr()
        st.w1_bf16 = self.pb["w1"].data_ptr()
        st.w2_bf16 = self.pb["w2"].data_ptr()
        st.step = self.steps
        return st

    def fit(self, data: "Dataset", steps: int, batch: int = 16384, lr: float = 3e-3, seed: int = 0) -> float:
        """Mini-batch Adam over the logged rows, all in the library
        (drt_mlp_train: targets, shuffle, learning-rate schedule and steps);
        returns the mean loss per step."""
        st = self.state()
        loss = torch.zeros(1, device=data.parts[0].x.device)
        self.ctx.mlp_train([p.record() for p in data.parts], st, steps, batch=batch, lr=lr, seed=seed, loss=loss)
        self.steps = int(st.step)
        return float(loss.item()) / max(1, steps)


@dataclasses.dataclass
class SceneLog:
    """One scene's logged training data (see drt_mlp_log)."""
    x: torch.Tensor        # [n, 32] bf16 bits of the segment features
    seg_log: torch.Tensor  # [n] logged sums of |w (f_u - f_l)| per segment
    seg_len: torch.Tensor  # [n] FP64 screen lengths of the segments
    n_samples: float       # primary edge samples behind seg_log

    def record(self) -> drt.MlpLog:
        return drt.MlpLog(self.x.data_ptr(), self.seg_log.data_ptr(), self.seg_len.data_ptr(), int(self.x.shape[0]),
                          float(self.n_samples))


@dataclasses.dataclass
class Dataset:
    parts: list  # SceneLog per logged scene

    @property
    def rows(self) -> int:
        return sum(int(p.x.shape[0]) for p in self.parts)


def _zero(n, dev):
    return torch.zeros(n, dtype=torch.float32, device=dev)


def collect(ctx: drt.Context, scene: drt.Scene, d_image: torch.Tensor, *, edge_spp: int, passes: int, seed: int,
            max_depth: int = 1) -> SceneLog:
    """Training data of one scene from the plain (length) distribution over
    its tile segments: `passes` backward passes of the primary edge term,
    each with edge_spp samples per pixel, logging |w (f_u - f_l)| per segment,
    and the segments' features."""
    dev = d_image.device
    _, _, _, seg_len = scene.segments()
    n = len(seg_len)
    log = _zero(n, dev)
    zeros = _zero(n, dev)
    dv = torch.zeros((scene.n_verts, 3), device=dev)
    for p in range(passes):
        o = drt.make_opts(1, edge_spp, max_depth=max_depth, seed=seed + p, terms=TERM_PRIMARY, seg_weights=zeros,
                          seg_log=log)
        scene.backward(d_image, o, d_verts=dv)
    n_samples = float(passes) * edge_spp * scene.width * scene.height
    x = torch.empty((n, N_IN), dtype=torch.int16, device=dev)
    scene.segment_features(d_image, x, step_image(scene, seed, max_depth))
    return SceneLog(x, log, torch.from_numpy(np.ascontiguousarray(seg_len, np.float64)).to(dev), n_samples)


IMAGE_SPP = 16


def step_image(scene: drt.Scene, seed: int, max_depth: int = 1) -> torch.Tensor:
    """The rendered image an optimisation step has before its backward pass
    (here IMAGE_SPP samples per pixel)."""
    img = torch.empty((scene.height, scene.width, 3), device="cuda")
    scene.render(img, drt.make_opts(IMAGE_SPP, IMAGE_SPP, max_depth=max_depth, seed=seed + 777))
    return img


# ---------------------------------------------------------------------------
# Evaluation: gradient variance x time against the plain sampler
# ---------------------------------------------------------------------------
@dataclasses.dataclass
class VarianceResult:
    var: float           # mean over vertex entries of Var_k(g_k), over the mean of gbar^2
    ms: float            # median milliseconds per gradient (proposal set-up included)
    mean: np.ndarray     # mean gradient [V*3]
    se: np.ndarray       # its standard error


def _summarise(runs: torch.Tensor, times, norm: float) -> VarianceResult:
    r = runs.double()
    k = r.shape[0]
    mean = r.mean(0)
    var = r.var(0, unbiased=True)
    return VarianceResult(float(var.mean()) / norm, float(np.median(times)), mean.cpu().numpy(),
                          (var / k).sqrt().cpu().numpy())


def gradient_runs(scene: drt.Scene, d_image: torch.Tensor, *, edge_spp: int, K: int, seed: int,
                  proposal: EdgeProposal | None = None, max_depth: int = 1, tape=None):
    """K primary-edge vertex gradients with independent seeds; per run the
    device time of the whole estimate (segment features, network and
    proposal CDF included for the learned proposal)."""
    dev = d_image.device
    runs = torch.zeros((K, scene.n_verts * 3), device=dev)
    times = []
    n = scene.num_segments() if proposal is not None else 0
    # the forward image the step rendered before its backward pass (not timed:
    # the plain sampler's step renders it too)
    image = step_image(scene, seed, max_depth) if proposal is not None else None
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for k in range(K):
        dv = runs[k].view(scene.n_verts, 3)
        e0.record()
        if proposal is not None:
            sc = proposal.scores(scene, d_image, n, image)
            o = drt.make_opts(1, edge_spp, max_depth=max_depth, seed=seed + k, terms=TERM_PRIMARY, seg_scores=sc)
        else:
            o = drt.make_opts(1, edge_spp, max_depth=max_depth, seed=seed + k, terms=TERM_PRIMARY)
        scene.backward(d_image, o, tape=tape, d_verts=dv)
        e1.record()
        e1.synchronize()
        times.append(e0.elapsed_time(e1))
    return runs, times


def compare(scene: drt.Scene, d_image: torch.Tensor, proposal: EdgeProposal, *, edge_spp: int, K: int, seed: int,
            max_depth: int = 1, warmup: int = 2):
    """Plain vs learned on one scene; returns (plain, learned, ratio, z2),
    ratio = (var_l ms_l) / (var_p ms_p), z2 = mean squared z-score of the
    difference of the two mean gradients (about 1 when both are unbiased)."""
    tape = None
    for prop in (None, proposal):  # warm-up (allocations, first launches)
        gradient_runs(scene, d_image, edge_spp=edge_spp, K=warmup, seed=seed + 10_000, proposal=prop,
                      max_depth=max_depth, tape=tape)
    rp, tp = gradient_runs(scene, d_image, edge_spp=edge_spp, K=K, seed=seed, proposal=None, max_depth=max_depth,
                           tape=tape)
    rl, tl = gradient_runs(scene, d_image, edge_spp=edge_spp, K=K, seed=seed + 50_000, proposal=proposal,
                           max_depth=max_depth, tape=tape)
    norm = float(((rp.double().mean(0) + rl.double().mean(0)) * 0.5).pow(2).mean())
    norm = norm if norm > 0 else 1.0
    plain = _summarise(rp, tp, norm)
    learned = _summarise(rl, tl, norm)
    ratio = (learned.var * learned.ms) / max(plain.var * plain.ms, 1e-30)
    se2 = plain.se ** 2 + learned.se ** 2
    ok = se2 > 0
    z2 = float(np.mean((plain.mean[ok] - learned.mean[ok]) ** 2 / se2[ok])) if ok.any() else 0.0
    return plain, learned, ratio, z2


# ---------------------------------------------------------------------------
# Train / evaluate protocol: network trained on logs of 16 direct-lighting
# scenes (icosphere of 5120 triangles, 256x256) and 4 procedural scenes
# (200k triangles, 512x512, depth 3); scored on 2 + 2 held-out scenes.
# ---------------------------------------------------------------------------
TRAIN_DIRECT = tuple(range(100, 116))
TRAIN_PROCEDURAL = tuple(range(116, 120))
HELD_OUT = ((200, "direct"), (201, "direct"), (202, "procedural"), (203, "procedural"))


def _make_scene(ctx, kind, seed):
    from . import scenegen as sg
    sc = sg.direct_lighting(seed) if kind == "direct" else sg.procedural(seed)
    s = drt.Scene.from_arrays(ctx, sc)
    w = torch.from_numpy(sg.loss_adjoint(seed, sc.width, sc.height)).cuda()
    return sc, s, w


def protocol(ctx: drt.Context, *, steps: int = 6000, k_direct: int = 32, k_procedural: int = 24,
             edge_spp_direct: int = 64, edge_spp_procedural: int = 32) -> dict:
    """Collect, train and evaluate; returns a JSON-ready summary with the
    learned/plain ratio of gradient variance x time per held-out scene and
    their geometric mean."""
    import time
    t0 = time.perf_counter()
    parts = []
    for seed in TRAIN_DIRECT:
        _, s, w = _make_scene(ctx, "direct", seed)
        parts.append(collect(ctx, s, w, edge_spp=16, passes=4, seed=seed * 1000))
        s.free()
    for seed in TRAIN_PROCEDURAL:
        _, s, w = _make_scene(ctx, "procedural", seed)
        parts.append(collect(ctx, s, w, edge_spp=4, passes=2, seed=seed * 1000, max_depth=3))
        s.free()
    data = Dataset(parts)
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    net = EdgeProposal(ctx, 0)
    loss_mean = net.fit(data, steps=steps)
    torch.cuda.synchronize()
    t2 = time.perf_counter()
    scenes = []
    for seed, kind in HELD_OUT:
        sc, s, w = _make_scene(ctx, kind, seed)
        direct = kind == "direct"
        es = edge_spp_direct if direct else edge_spp_procedural
        md = 1 if direct else 3
        plain, learned, ratio, z2 = compare(s, w, net, edge_spp=es, K=k_direct if direct else k_procedural,
                                            seed=seed * 7, max_depth=md)
        scenes.append({"scene": "%s seed %d" % (kind, seed), "triangles": int(len(sc.tris)),
                       "width": sc.width, "height": sc.height, "max_depth": md, "edge_spp": es,
                       "runs": k_direct if direct else k_procedural, "var_plain": plain.var,
                       "var_learned": learned.var, "ms_plain": plain.ms, "ms_learned": learned.ms,
                       "ratio": ratio, "mean_z2": z2})
        s.free()
    code, info = ctx.check_device()
    if code != 0:
        raise RuntimeError("device error flag %d (%d) in the proposal protocol" % (code, info))
    gm = float(np.exp(np.mean([np.log(max(r["ratio"], 1e-30)) for r in scenes])))
    return {"ratio_geomean": gm, "ratio_unit": "learned/plain gradient variance x time (<1: learned wins)",
            "scenes": scenes, "train_rows": data.rows, "train_steps": steps,
            "collect_s": t1 - t0, "train_s": t2 - t1, "loss_mean": loss_mean,
            "variance": "mean over vertex entries of the run variance of the primary edge gradient, "
                        "over the mean squared gradient",
            "time": "median device ms of one gradient estimate; learned includes segment features, network "
                    "forward and proposal CDF"}
