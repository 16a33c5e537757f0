"""Python binding of the C ABI in include/drt.h (argument marshalling only).

Every step of rendering and differentiation runs in the CUDA library
``_lib/libdrt.so``; this module passes pointers, sizes and the current CUDA
stream.  There is no fallback: if the library cannot be loaded, every call
raises.

Arrays may be torch CUDA tensors, torch CPU tensors or numpy arrays (host
memory is copied by the library on the stream).
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

DRT_OK = 0
STATUS = {0: "OK", 1: "INVALID_ARG", 2: "CUDA", 3: "OOM", 4: "TIMEOUT", 5: "DEVICE_FLAG", 6: "STATE"}
TERM_INTERIOR, TERM_PRIMARY, TERM_SECONDARY = 1, 2, 4
AOV_ALBEDO, AOV_POSITION, AOV_NORMAL, AOV_DEPTH = 1, 2, 3, 4

EXPORTED = ("drt_create", "drt_destroy", "drt_scene_upload", "drt_scene_update_vertices", "drt_scene_update_params",
            "drt_scene_free", "drt_render", "drt_render_backward", "drt_tape_free", "drt_check_device",
            "drt_last_error", "drt_version", "drt_debug_closest", "drt_profile_enable", "drt_profile_read",
            "drt_counters_enable", "drt_counters_read", "drt_render_backward_noalloc", "drt_scene_segments",
            "drt_mlp_forward", "drt_mlp_backward", "drt_adam_step", "drt_segment_features", "drt_batch_create",
            "drt_batch_run", "drt_batch_get_info", "drt_batch_free", "drt_render_batch", "drt_probe_fma",
            "drt_probe_l2", "drt_mlp_train")
BATCH_PASSES = ("render", "interior", "secondary", "path", "primary")


class DrtError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("drt status %s: %s" % (STATUS.get(status, status), msg))
        self.status = status


class SceneDesc(ctypes.Structure):
    _fields_ = [("verts", ctypes.c_void_p), ("n_verts", ctypes.c_int32), ("tris", ctypes.c_void_p),
                ("n_tris", ctypes.c_int32), ("albedo", ctypes.c_void_p), ("light_tris", ctypes.c_void_p),
                ("n_light_tris", ctypes.c_int32), ("radiance", ctypes.c_void_p), ("cam_to_world", ctypes.c_void_p),
                ("cam_scale", ctypes.c_float), ("cam_type", ctypes.c_int32), ("width", ctypes.c_int32),
                ("height", ctypes.c_int32), ("bvh_leaf_size", ctypes.c_int32)]


class RenderOpts(ctypes.Structure):
    _fields_ = [("spp", ctypes.c_int32), ("edge_spp", ctypes.c_int32), ("max_depth", ctypes.c_int32),
                ("primary_only", ctypes.c_int32), ("seed", ctypes.c_uint64), ("eps_rel", ctypes.c_float),
                ("terms", ctypes.c_int32), ("proposal", ctypes.c_int32), ("seg_weights", ctypes.c_void_p),
                ("n_seg_weights", ctypes.c_int64), ("seg_log", ctypes.c_void_p), ("scene_id", ctypes.c_int32),
                ("sec_sampler", ctypes.c_int32), ("sec_tree_samples", ctypes.c_int32), ("sec_point", ctypes.c_int32),
                ("pix_begin", ctypes.c_int32), ("pix_end", ctypes.c_int32), ("edge_begin", ctypes.c_int64),
                ("edge_end", ctypes.c_int64), ("aov", ctypes.c_int32), ("sec_nee", ctypes.c_int32),
                ("nee_width", ctypes.c_float), ("spp_per_pass", ctypes.c_int32)]


class MlpWeights(ctypes.Structure):
    _fields_ = [("w1", ctypes.c_void_p), ("b1", ctypes.c_void_p), ("w2", ctypes.c_void_p), ("b2", ctypes.c_void_p),
                ("w3", ctypes.c_void_p), ("b3", ctypes.c_void_p)]


class MlpGrads(ctypes.Structure):
    _fields_ = [("w1", ctypes.c_void_p), ("b1", ctypes.c_void_p), ("w2", ctypes.c_void_p), ("b2", ctypes.c_void_p),
                ("w3", ctypes.c_void_p), ("b3", ctypes.c_void_p)]


class MlpLog(ctypes.Structure):
    _fields_ = [("x", ctypes.c_void_p), ("seg_log", ctypes.c_void_p), ("seg_len", ctypes.c_void_p),
                ("n", ctypes.c_int64), ("n_samples", ctypes.c_double)]


class MlpState(ctypes.Structure):
    _fields_ = [("p", ctypes.c_void_p * 6), ("m1", ctypes.c_void_p * 6), ("m2", ctypes.c_void_p * 6),
                ("g", ctypes.c_void_p * 6), ("w1_bf16", ctypes.c_void_p), ("w2_bf16", ctypes.c_void_p),
                ("step", ctypes.c_int64)]


class MlpTrainOpts(ctypes.Structure):
    _fields_ = [("steps", ctypes.c_int32), ("batch", ctypes.c_int32), ("lr", ctypes.c_float),
                ("delta", ctypes.c_float), ("seed", ctypes.c_uint64), ("loss", ctypes.c_void_p),
                ("rows_target", ctypes.c_void_p), ("rows_mask", ctypes.c_void_p), ("rows_index", ctypes.c_void_p)]


class Grads(ctypes.Structure):
    _fields_ = [("d_verts", ctypes.c_void_p), ("d_albedo", ctypes.c_void_p), ("d_radiance", ctypes.c_void_p),
                ("d_cam_to_world", ctypes.c_void_p), ("d_cam_scale", ctypes.c_void_p),
                ("dimage_dparam", ctypes.c_void_p), ("n_jac", ctypes.c_int32), ("pad_", ctypes.c_int32),
                ("jac_param", ctypes.c_int64 * 8)]


class BatchItem(ctypes.Structure):
    _fields_ = [("scene", ctypes.c_void_p), ("image", ctypes.c_void_p), ("d_image", ctypes.c_void_p),
                ("grads", Grads), ("verts", ctypes.c_void_p)]


class BatchInfo(ctypes.Structure):
    _fields_ = [("ctas_per_sm", ctypes.c_int32 * 5), ("grid", ctypes.c_int32 * 5), ("chunk", ctypes.c_int32 * 5),
                ("edge_per_thread_mult", ctypes.c_int32), ("graph", ctypes.c_int32), ("tuned", ctypes.c_int32),
                ("items", ctypes.c_int64 * 5), ("edge_samples", ctypes.c_int64), ("tune_ms", ctypes.c_double)]


_LIB = None


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load libdrt.so (building it first if needed); raises if unavailable."""
    global _LIB
    if _LIB is not None:
        return _LIB
    path = _build.LIB
    if not os.path.exists(path) or not _build.up_to_date():
        if not build_if_missing:
            raise RuntimeError("CUDA library %s is missing; run __graft_entry__.build()" % path)
        _build.build()
    lib = ctypes.CDLL(path)
    vp, i32, u64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_uint64
    pp = ctypes.POINTER(ctypes.c_void_p)
    sig = {
        "drt_create": ([ctypes.c_int, pp], i32),
        "drt_destroy": ([vp], i32),
        "drt_scene_upload": ([vp, ctypes.POINTER(SceneDesc), vp, pp], i32),
        "drt_scene_update_vertices": ([vp, vp, vp, vp], i32),
        "drt_scene_update_params": ([vp, vp, vp, vp, vp, vp, vp], i32),
        "drt_scene_free": ([vp, vp], i32),
        "drt_render": ([vp, vp, ctypes.POINTER(RenderOpts), vp, pp, vp], i32),
        "drt_render_backward": ([vp, vp, vp, ctypes.POINTER(RenderOpts), vp, ctypes.POINTER(Grads), vp], i32),
        "drt_tape_free": ([vp, vp], i32),
        "drt_mlp_forward": ([vp, vp, ctypes.c_int64, ctypes.POINTER(MlpWeights), vp, vp], i32),
        "drt_mlp_backward": ([vp, vp, vp, vp, ctypes.c_int64, ctypes.c_float, ctypes.POINTER(MlpWeights),
                              ctypes.POINTER(MlpGrads), vp, vp], i32),
        "drt_adam_step": ([vp, vp, vp, vp, vp, vp, ctypes.c_int64, ctypes.c_float, ctypes.c_float, ctypes.c_float,
                           ctypes.c_float, ctypes.c_int32, vp], i32),
        "drt_segment_features": ([vp, vp, vp, vp, vp, vp], i32),
        "drt_scene_segments": ([vp, vp, ctypes.POINTER(ctypes.c_int64), vp, vp, vp, ctypes.c_int64, vp], i32),
        "drt_render_backward_noalloc": ([vp, vp, vp, ctypes.POINTER(RenderOpts), vp, ctypes.POINTER(Grads), vp],
                                        i32),
        "drt_check_device": ([vp, vp, ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int32)], i32),
        "drt_debug_closest": ([vp, vp, ctypes.c_int64, vp, vp, vp, vp, vp], i32),
        "drt_profile_enable": ([vp, ctypes.c_int], i32),
        "drt_profile_read": ([vp, ctypes.c_int, vp, vp, vp, ctypes.POINTER(ctypes.c_int)], i32),
        "drt_counters_enable": ([vp, ctypes.c_int], i32),
        "drt_counters_read": ([vp, vp], i32),
        "drt_batch_create": ([vp, ctypes.POINTER(BatchItem), i32, ctypes.POINTER(RenderOpts), i32, i32, pp], i32),
        "drt_batch_run": ([vp, vp, vp], i32),
        "drt_batch_get_info": ([vp, vp, ctypes.POINTER(BatchInfo)], i32),
        "drt_batch_free": ([vp, vp], i32),
        "drt_render_batch": ([vp, pp, i32, ctypes.POINTER(RenderOpts), pp, pp, ctypes.POINTER(Grads), vp], i32),
        "drt_mlp_train": ([vp, ctypes.POINTER(MlpLog), i32, ctypes.POINTER(MlpTrainOpts), ctypes.POINTER(MlpState),
                           vp], i32),
        "drt_probe_fma": ([vp, ctypes.POINTER(ctypes.c_double), vp], i32),
        "drt_probe_l2": ([vp, ctypes.c_int64, ctypes.POINTER(ctypes.c_double), vp], i32),
        "drt_last_error": ([vp], ctypes.c_char_p),
        "drt_version": ([], ctypes.c_char_p),
    }
    for name, (args, res) in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = res
    _LIB = lib
    return lib


def _check(status):
    if status != DRT_OK:
        raise DrtError(status, load().drt_last_error(None).decode(errors="replace"))


def _ptr(a):
    """Pointer of a torch tensor or numpy array (must stay alive during the call)."""
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("array must be contiguous")
        return a.data_ptr()
    if isinstance(a, np.ndarray):
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        return a.ctypes.data
    raise TypeError("unsupported array type %r" % type(a))


def _stream(stream):
    if stream is not None:
        return stream
    try:
        import torch
        if torch.cuda.is_available():
            return torch.cuda.current_stream().cuda_stream
    except Exception:
        pass
    return 0


def make_opts(spp, edge_spp=None, max_depth=1, primary_only=False, seed=0, eps_rel=0.0, terms=0,
              seg_weights=None, seg_log=None, seg_scores=None, scene_id=0, sec_tree_samples=0,
              sec_point=0, pixels=None, edges=None, aov=0, sec_nee=0, nee_width=0.0, spp_per_pass=0) -> RenderOpts:
    """seg_weights: a CUDA float32 tensor of per-segment weights selects the
    mixture proposal 1; seg_scores: per-segment network scores select the
    mixture proposal 2.  The tensor must stay alive until the backward call
    returns.  sec_tree_samples > 0 picks secondary edges through the edge
    hierarchy with that many root samples (0: by 3D length).  sec_point=1
    samples the point on a secondary edge by the clamped-cosine density over
    the edge's arc mixed with uniform (0: uniform).  pixels=(begin, end) and
    edges=(begin, end) restrict the backward pass to the interior and
    secondary samples of those pixels and to those primary edge samples
    (default: all).  aov: geometry buffer of the first hit (AOV_ALBEDO,
    AOV_POSITION, AOV_NORMAL, AOV_DEPTH; 0: the image).  sec_nee=1 adds
    next-event estimation for edges (Sec. 5.3.3) beside the length sampler,
    with billboards of width nee_width (<= 0: derived from the vertices).
    spp_per_pass = k (0 < k < spp, spp a multiple of k) renders and
    differentiates the interior samples in spp / k passes of k samples per
    pixel with the Philox keys seed + p 0x9E3779B97F4A7C15, so the tape
    holds one pass."""
    if seg_weights is not None and seg_scores is not None:
        raise ValueError("give seg_weights or seg_scores, not both")
    mode, w = (1, seg_weights) if seg_weights is not None else ((2, seg_scores) if seg_scores is not None else (0, None))
    n = int(w.numel()) if w is not None else 0
    return RenderOpts(int(spp), int(spp if edge_spp is None else edge_spp), int(max_depth),
                      int(bool(primary_only) or aov > 0),
                      int(seed) & (2 ** 64 - 1), float(eps_rel), int(terms), mode,
                      _ptr(w) if w is not None else None, n,
                      _ptr(seg_log) if seg_log is not None else None, int(scene_id),
                      1 if sec_tree_samples > 0 else 0, int(sec_tree_samples), int(sec_point),
                      int(pixels[0]) if pixels else 0, int(pixels[1]) if pixels else 0,
                      int(edges[0]) if edges else 0, int(edges[1]) if edges else 0, int(aov), int(sec_nee),
                      float(nee_width), int(spp_per_pass))


class Context:
    """A library context on one CUDA device."""

    def __init__(self, device: int = 0):
        self.lib = load()
        h = ctypes.c_void_p()
        _check(self.lib.drt_create(int(device), ctypes.byref(h)))
        self.handle = h

    def close(self):
        if self.handle:
            self.lib.drt_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def check_device(self, stream=None):
        """Synchronise and read the device error flag; returns (code, info)."""
        code, info = ctypes.c_int32(), ctypes.c_int32()
        st = self.lib.drt_check_device(self.handle, _stream(stream), ctypes.byref(code), ctypes.byref(info))
        if st not in (DRT_OK, 5):
            _check(st)
        return code.value, info.value


    def profile(self, enable: bool):
        """Bracket every library kernel launch with CUDA events on its stream."""
        _check(self.lib.drt_profile_enable(self.handle, int(bool(enable))))

    def profile_read(self):
        """{kernel name: (total ms, launches)} since the last read (synchronises)."""
        mx = 128
        names = ctypes.create_string_buffer(64 * mx)
        ms = np.zeros(mx, np.float64)
        ln = np.zeros(mx, np.int64)
        n = ctypes.c_int()
        _check(self.lib.drt_profile_read(self.handle, mx, names, ms.ctypes.data, ln.ctypes.data, ctypes.byref(n)))
        out = {}
        for i in range(n.value):
            nm = names.raw[64 * i:64 * (i + 1)].split(b"\0")[0].decode()
            out[nm] = (float(ms[i]), int(ln[i]))
        return out

    def counters(self, enable: bool):
        _check(self.lib.drt_counters_enable(self.handle, int(bool(enable))))

    COUNTER_SLOTS = ("render", "backward_interior", "backward_primary_edges", "debug", "backward_secondary_edges",
                     "backward_secondary_sides", "backward_secondary_bounce", "backward_primary_bounce",
                     "render_bounce")

    def counters_read(self):
        """{slot: dict(closest_rays, shadow_rays, nodes, tris)} (synchronises, resets)."""
        a = np.zeros((len(self.COUNTER_SLOTS), 4), np.int64)
        _check(self.lib.drt_counters_read(self.handle, a.ctypes.data))
        return {nm: dict(closest_rays=int(a[i, 0]), shadow_rays=int(a[i, 1]), nodes=int(a[i, 2]), tris=int(a[i, 3]))
                for i, nm in enumerate(self.COUNTER_SLOTS)}


    def probe_fma(self, stream=None) -> float:
        """Measured FP32 FMA lane-operations per second (synchronises)."""
        v = ctypes.c_double()
        _check(self.lib.drt_probe_fma(self.handle, ctypes.byref(v), _stream(stream)))
        return v.value

    def probe_l2(self, nbytes=32 << 20, stream=None) -> float:
        """Measured L2 copy bandwidth in bytes/s over nbytes of buffers (synchronises)."""
        v = ctypes.c_double()
        _check(self.lib.drt_probe_l2(self.handle, int(nbytes), ctypes.byref(v), _stream(stream)))
        return v.value

    def mlp_forward(self, x, w: "MlpWeights", y, stream=None):
        """y [m] = network(x [m,32] bf16); w holds device pointers."""
        _check(self.lib.drt_mlp_forward(self.handle, _ptr(x), int(x.shape[0]), ctypes.byref(w), _ptr(y),
                                        _stream(stream)))

    def mlp_backward(self, x, target, mask, inv_n, w: "MlpWeights", g: "MlpGrads", loss, stream=None):
        _check(self.lib.drt_mlp_backward(self.handle, _ptr(x), _ptr(target), _ptr(mask), int(x.shape[0]),
                                         float(inv_n), ctypes.byref(w), ctypes.byref(g), _ptr(loss),
                                         _stream(stream)))

    def mlp_train(self, logs, state: "MlpState", steps, batch=0, lr=0.0, delta=0.0, seed=0, loss=None,
                  rows_target=None, rows_mask=None, rows_index=None, stream=None):
        """drt_mlp_train over a sequence of MlpLog records (their arrays must
        stay alive during the call); state is updated in place."""
        arr = (MlpLog * len(logs))(*logs)
        o = MlpTrainOpts(int(steps), int(batch), float(lr), float(delta), int(seed) & (2 ** 64 - 1), _ptr(loss),
                         _ptr(rows_target), _ptr(rows_mask), _ptr(rows_index))
        _check(self.lib.drt_mlp_train(self.handle, arr, len(logs), ctypes.byref(o), ctypes.byref(state),
                                      _stream(stream)))

    def adam_step(self, params, grads, m1, m2, params_bf16, lr, step, beta1=0.9, beta2=0.999, eps=1e-8,
                  stream=None):
        _check(self.lib.drt_adam_step(self.handle, _ptr(params), _ptr(grads), _ptr(m1), _ptr(m2),
                                      _ptr(params_bf16), int(params.numel()), float(lr), float(beta1), float(beta2),
                                      float(eps), int(step), _stream(stream)))


class Tape:
    def __init__(self, ctx, handle):
        self.ctx, self.handle = ctx, handle

    def free(self):
        if self.handle:
            self.ctx.lib.drt_tape_free(self.ctx.handle, self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


class Scene:
    """An uploaded scene.  ``arrays`` are kept alive until the upload returns."""

    def __init__(self, ctx: Context, verts, tris, albedo, light_tris, radiance, cam_to_world, cam_scale, cam_type,
                 width, height, stream=None, bvh_leaf_size=0):
        self.ctx = ctx
        self.n_verts, self.n_tris = int(verts.shape[0]), int(tris.shape[0])
        self.width, self.height = int(width), int(height)
        nl = int(light_tris.shape[0]) if light_tris is not None else 0
        desc = SceneDesc(_ptr(verts), self.n_verts, _ptr(tris), self.n_tris, _ptr(albedo),
                         _ptr(light_tris) if nl else None, nl, _ptr(radiance), _ptr(cam_to_world),
                         float(cam_scale), int(cam_type), self.width, self.height, int(bvh_leaf_size))
        h = ctypes.c_void_p()
        _check(ctx.lib.drt_scene_upload(ctx.handle, ctypes.byref(desc), _stream(stream), ctypes.byref(h)))
        self.handle = h

    @classmethod
    def from_arrays(cls, ctx, sc, stream=None, bvh_leaf_size=0):
        """Upload a ``scenegen.Scene`` (host numpy arrays)."""
        return cls(ctx, sc.verts, sc.tris, sc.albedo, sc.light_tris, sc.radiance, sc.cam_to_world, sc.cam_scale,
                   sc.cam_type, sc.width, sc.height, stream, bvh_leaf_size)

    def update_vertices(self, verts, stream=None):
        _check(self.ctx.lib.drt_scene_update_vertices(self.ctx.handle, self.handle, _ptr(verts), _stream(stream)))

    def update_params(self, albedo=None, radiance=None, cam_to_world=None, cam_scale=None, stream=None):
        cs = None
        if cam_scale is not None:
            cs = np.array([cam_scale], np.float32) if np.isscalar(cam_scale) else cam_scale
        _check(self.ctx.lib.drt_scene_update_params(self.ctx.handle, self.handle, _ptr(albedo), _ptr(radiance),
                                                    _ptr(cam_to_world), _ptr(cs), _stream(stream)))

    def free(self):
        if self.handle:
            self.ctx.lib.drt_scene_free(self.ctx.handle, self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass

    def segments(self, stream=None):
        """Tile segments of the clipped primary edges as numpy arrays:
        (edge, tile) int32, (s0, s1) float32, lengths float64."""
        n = ctypes.c_int64()
        _check(self.ctx.lib.drt_scene_segments(self.ctx.handle, self.handle, ctypes.byref(n), None, None, None, 0,
                                               _stream(stream)))
        et = np.zeros((n.value, 2), np.int32)
        s01 = np.zeros((n.value, 2), np.float32)
        ln = np.zeros(n.value, np.float64)
        _check(self.ctx.lib.drt_scene_segments(self.ctx.handle, self.handle, ctypes.byref(n), _ptr(et), _ptr(s01),
                                               _ptr(ln), n.value, _stream(stream)))
        return et[:, 0], et[:, 1], s01, ln

    def num_segments(self, stream=None) -> int:
        """Number of tile segments of the current clipped primary edges."""
        n = ctypes.c_int64()
        _check(self.ctx.lib.drt_scene_segments(self.ctx.handle, self.handle, ctypes.byref(n), None, None, None, 0,
                                               _stream(stream)))
        return n.value

    def segment_features(self, d_image, x, image=None, stream=None):
        """Features [n_seg, 32] (bf16 device tensor x) of the current segments;
        ``image`` is the step's rendered image (optional)."""
        _check(self.ctx.lib.drt_segment_features(self.ctx.handle, self.handle, _ptr(d_image), _ptr(image),
                                                 _ptr(x), _stream(stream)))

    def closest(self, o, d, tri, tb, stream=None):
        """Closest hits of rays o, d [n,3] into tri [n] (int32) and tb [n,3]."""
        _check(self.ctx.lib.drt_debug_closest(self.ctx.handle, self.handle, int(o.shape[0]), _ptr(o), _ptr(d),
                                              _ptr(tri), _ptr(tb), _stream(stream)))

    def render(self, image, opts: RenderOpts, want_tape=False, stream=None, reuse=None):
        """Render into ``image`` [H,W,3] float32; returns a Tape if asked.
        ``reuse``: a Tape of this scene whose storage is overwritten."""
        if reuse is not None:
            th = reuse.handle
            _check(self.ctx.lib.drt_render(self.ctx.handle, self.handle, ctypes.byref(opts), _ptr(image),
                                           ctypes.byref(th), _stream(stream)))
            reuse.handle = th
            return reuse
        th = ctypes.c_void_p()
        _check(self.ctx.lib.drt_render(self.ctx.handle, self.handle, ctypes.byref(opts), _ptr(image),
                                       ctypes.byref(th) if want_tape else None, _stream(stream)))
        return Tape(self.ctx, th) if want_tape else None

    def backward_noalloc(self, d_image, opts: RenderOpts, tape=None, d_verts=None, d_albedo=None, d_radiance=None,
                         d_cam_to_world=None, d_cam_scale=None, stream=None):
        """``backward`` for callers that cannot allocate device memory during
        the call: device arrays only, scratch in a fixed array inside the
        library (see drt_render_backward_noalloc in include/drt.h)."""
        g = Grads(_ptr(d_verts), _ptr(d_albedo), _ptr(d_radiance), _ptr(d_cam_to_world), _ptr(d_cam_scale))
        _check(self.ctx.lib.drt_render_backward_noalloc(self.ctx.handle, self.handle, tape.handle if tape else None,
                                                        ctypes.byref(opts), _ptr(d_image), ctypes.byref(g),
                                                        _stream(stream)))

    def backward(self, d_image, opts: RenderOpts, tape=None, d_verts=None, d_albedo=None, d_radiance=None,
                 d_cam_to_world=None, d_cam_scale=None, dimage_dparam=None, jac_params=None, stream=None):
        """Add d loss / d parameters into the given gradient arrays;
        dimage_dparam [n, H, W] with jac_params (n <= 8 flat parameter
        indices) also receives the per-pixel gradient image."""
        g = Grads(_ptr(d_verts), _ptr(d_albedo), _ptr(d_radiance), _ptr(d_cam_to_world), _ptr(d_cam_scale))
        if dimage_dparam is not None:
            idx = [int(i) for i in (jac_params or [])]
            g.dimage_dparam = _ptr(dimage_dparam)
            g.n_jac = len(idx)
            for k, i in enumerate(idx[:8]):
                g.jac_param[k] = i
        _check(self.ctx.lib.drt_render_backward(self.ctx.handle, self.handle, tape.handle if tape else None,
                                                ctypes.byref(opts), _ptr(d_image), ctypes.byref(g),
                                                _stream(stream)))


def _grads_of(g):
    g = g or {}
    return Grads(_ptr(g.get("d_verts")), _ptr(g.get("d_albedo")), _ptr(g.get("d_radiance")),
                 _ptr(g.get("d_cam_to_world")), _ptr(g.get("d_cam_scale")))


class Batch:
    """Many scenes rendered and differentiated per step (drt_batch_* in
    include/drt.h).  images[k], d_images[k] (or None), grads[k] (a dict of
    gradient tensors, or None) and verts[k] (or None) are device tensors that
    must stay alive with the batch; scene k samples with scene_id k."""

    def __init__(self, ctx: Context, scenes, images, opts: RenderOpts, d_images=None, grads=None, verts=None,
                 use_graph=True, autotune=True):
        n = len(scenes)
        self.ctx, self.handle = ctx, None
        self._keep = (list(scenes), list(images), d_images, grads, verts, opts)
        arr = (BatchItem * n)()
        for k in range(n):
            arr[k].scene = scenes[k].handle.value
            arr[k].image = _ptr(images[k])
            arr[k].d_image = _ptr(d_images[k]) if d_images is not None else None
            arr[k].grads = _grads_of(grads[k] if grads is not None else None)
            arr[k].verts = _ptr(verts[k]) if verts is not None else None
        h = ctypes.c_void_p()
        _check(ctx.lib.drt_batch_create(ctx.handle, arr, n, ctypes.byref(opts), int(bool(use_graph)),
                                        int(bool(autotune)), ctypes.byref(h)))
        self.handle = h

    def run(self, stream=None):
        _check(self.ctx.lib.drt_batch_run(self.ctx.handle, self.handle, _stream(stream)))

    def info(self) -> dict:
        i = BatchInfo()
        _check(self.ctx.lib.drt_batch_get_info(self.ctx.handle, self.handle, ctypes.byref(i)))
        per = {nm: dict(ctas_per_sm=i.ctas_per_sm[p], grid=i.grid[p], chunk=i.chunk[p], items=i.items[p])
               for p, nm in enumerate(BATCH_PASSES)}
        return dict(passes=per, edge_per_thread_mult=i.edge_per_thread_mult, graph=bool(i.graph),
                    tuned=bool(i.tuned), edge_samples=i.edge_samples, tune_ms=i.tune_ms)

    def free(self):
        if self.handle:
            self.ctx.lib.drt_batch_free(self.ctx.handle, self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def render_batch(ctx: Context, scenes, images, opts: RenderOpts, d_images=None, grads=None, stream=None):
    """One-shot batch (no graph, no tuning); synchronises the stream."""
    n = len(scenes)
    sc = (ctypes.c_void_p * n)(*[s.handle.value for s in scenes])
    im = (ctypes.c_void_p * n)(*[_ptr(x) for x in images])
    di = (ctypes.c_void_p * n)(*[_ptr(x) for x in d_images]) if d_images is not None else None
    gr = (Grads * n)(*[_grads_of(g) for g in grads]) if grads is not None else None
    _check(ctx.lib.drt_render_batch(ctx.handle, sc, n, ctypes.byref(opts), im, di, gr, _stream(stream)))
