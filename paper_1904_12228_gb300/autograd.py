"""PyTorch autograd interface (Sec. 5.4: scenes as tensors, gradients flowing
back into them).

``Renderer`` owns an uploaded scene of fixed topology.  Calling it with
parameter tensors renders an image whose backward pass runs the library's
``drt_render_backward``: the interior adjoint over the checkpointed path and
the primary and secondary edge samples.  Every step runs in the CUDA library;
this module only moves tensors.

One forward is paired with one backward: the library refuses (DRT_ERR_STATE)
a backward whose scene changed since its forward.
"""
from __future__ import annotations

import torch

from . import drt


class _RenderFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, verts, albedo, radiance, cam_to_world, cam_scale, renderer):
        S = renderer.scene
        S.update_vertices(verts.detach().contiguous())
        S.update_params(albedo=albedo.detach().contiguous(), radiance=radiance.detach().contiguous(),
                        cam_to_world=cam_to_world.detach().contiguous(), cam_scale=cam_scale.detach().contiguous())
        opts = renderer.next_opts()
        image = torch.empty((renderer.height, renderer.width, 3), dtype=torch.float32, device=verts.device)
        renderer.tape = S.render(image, opts, want_tape=True, reuse=renderer.tape)
        ctx.renderer, ctx.opts = renderer, opts
        ctx.shapes = (verts.shape, albedo.shape)
        return image

    @staticmethod
    def backward(ctx, d_image):
        r = ctx.renderer
        dev = d_image.device
        dv = torch.zeros(ctx.shapes[0], dtype=torch.float32, device=dev)
        da = torch.zeros(ctx.shapes[1], dtype=torch.float32, device=dev)
        dr = torch.zeros(3, dtype=torch.float32, device=dev)
        dc = torch.zeros((4, 4), dtype=torch.float32, device=dev)
        ds = torch.zeros(1, dtype=torch.float32, device=dev)
        r.scene.backward(d_image.contiguous(), ctx.opts, tape=r.tape, d_verts=dv, d_albedo=da, d_radiance=dr,
                         d_cam_to_world=dc[:3], d_cam_scale=ds)
        return dv, da, dr, dc, ds, None


class Renderer:
    """Differentiable renderer of one scene (fixed triangles and lights).

    spp / edge_spp / max_depth / eps_rel follow drt_render_opts; each call
    uses a fresh seed (seed, seed+1, ...) so gradients are independent.
    """

    def __init__(self, scene, device: int = 0, spp: int = 4, edge_spp: int | None = None, max_depth: int = 1,
                 seed: int = 0, ctx: drt.Context | None = None):
        self.ctx = ctx or drt.Context(device)
        self.scene = drt.Scene.from_arrays(self.ctx, scene)
        self.width, self.height = scene.width, scene.height
        self.spp, self.edge_spp = spp, spp if edge_spp is None else edge_spp
        self.max_depth = max_depth
        self.seed = seed
        self.tape = None

    def next_opts(self):
        o = drt.make_opts(self.spp, self.edge_spp, max_depth=self.max_depth, seed=self.seed)
        self.seed += 1
        return o

    def __call__(self, verts, albedo, radiance, cam_to_world, cam_scale):
        """Image [H,W,3] of the scene with these parameters (CUDA tensors:
        verts [V,3], albedo [T,3], radiance [3], cam_to_world [4,4],
        cam_scale [1])."""
        return _RenderFn.apply(verts, albedo, radiance, cam_to_world, cam_scale, self)
