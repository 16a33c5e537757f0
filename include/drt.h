/*
 * drt.h -- C ABI of the GB300 differentiable Monte Carlo ray tracer with edge
 * sampling (T.-M. Li, "Differentiable Visual Computing", Chapter 5).
 *
 * The library renders a triangle-mesh scene by Monte Carlo ray tracing and
 * returns the gradient of a scalar loss of the image with respect to vertex
 * positions, per-triangle albedo, light radiance and camera (the problem
 * statement of Sec. 5.2).  The gradient is the sum of
 *   - the interior term: reverse-mode derivative of the per-sample integrand
 *     (second integral of Eq. redner_product_rule), and
 *   - the edge terms: explicitly sampled points on triangle edges, the
 *     radiance difference across each edge (Eq. dirac_rewrite, Eq. mc for
 *     primary visibility; Eq. dirac_3d, Eq. dirac_3d_edge, Eq. alpha_3d for
 *     shadows and indirect light).
 *
 * Conventions shared by every call
 *   - Pointers to arrays may be device memory or host memory; the library
 *     checks each with cudaPointerGetAttributes.  Host inputs are copied to the
 *     device on `stream`; when an OUTPUT pointer is host memory the call
 *     synchronises `stream` before returning so the data is there.  The device
 *     staging buffers of host arrays are kept per device for later calls
 *     (at most 16) and released by drt_destroy.
 *   - `stream` is a cudaStream_t (NULL = legacy default stream).  All device
 *     work of a call is enqueued on it, in order.
 *   - Arrays are C-order float32 / int32 unless stated.  Images are [H,W,3],
 *     row 0 at the top of the view.
 *   - Every call returns a drt_status; none throws.  drt_last_error(ctx)
 *     gives a message for the last failing call on this thread.
 *   - Objects (context, scene, tape) are owned by the library and freed with
 *     the matching *_free / drt_destroy call.  Caller arrays are borrowed for
 *     the duration of the call only; the library keeps its own copies.
 */
#ifndef DRT_H
#define DRT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  DRT_OK = 0,
  DRT_ERR_INVALID_ARG = 1, /* bad size, index, NaN/Inf input, NULL where not allowed */
  DRT_ERR_CUDA = 2,        /* a CUDA runtime call failed (message has the CUDA error) */
  DRT_ERR_OOM = 3,         /* device allocation failed */
  DRT_ERR_TIMEOUT = 4,     /* a bounded device wait gave up */
  DRT_ERR_DEVICE_FLAG = 5, /* a kernel raised the device error flag (see drt_check_device) */
  DRT_ERR_STATE = 6        /* call out of order (e.g. backward with a tape of another scene) */
} drt_status;

/* Device error-flag codes, read back by drt_check_device. */
enum {
  DRT_DEV_OK = 0,
  DRT_DEV_STACK_OVERFLOW = 1,  /* traversal stack full: a subtree was skipped (info = node) */
  DRT_DEV_NONFINITE_INPUT = 2, /* NaN/Inf vertex coordinate (info = flat index) */
  DRT_DEV_BAD_INDEX = 3,       /* out-of-range index met on the device */
  DRT_DEV_TRAVERSAL_CAP = 4,   /* traversal visited more nodes than the tree has (malformed BVH) */
  DRT_DEV_REFIT_CAP = 5,       /* BVH refit climbed more levels than there are nodes */
  DRT_DEV_TIMEOUT = 6          /* a bounded wait (tensor-core completion barrier) gave up (info = block) */
};

typedef struct drt_context drt_context;
typedef struct drt_scene drt_scene;
typedef struct drt_tape drt_tape;
typedef struct drt_batch drt_batch;

/* Cameras: orthographic and pinhole map 3D lines to screen lines, so their
 * primary edges are sampled on the projected segments (Sec. 5.2.1).  The
 * equidistant fisheye (Sec. 5.2, "Cameras with Non-linear Projections")
 * sends the screen point at distance r from the image centre, in units of
 * half the image height, along the direction at angle r * cam_scale from
 * the optical axis; its primary edges are sampled in 3D (by their chord on
 * the unit sphere of directions from the camera), and each sample's edge
 * term follows the curved image of the edge.  A fisheye scene needs
 * cam_scale * sqrt((W/H)^2 + 1) < 0.99 pi (every pixel sees a direction);
 * it takes the length proposal only and no batch. */
enum { DRT_CAMERA_ORTHO = 0, DRT_CAMERA_PINHOLE = 1, DRT_CAMERA_FISHEYE = 2 };

/* A scene given as flat arrays, the way Sec. 5.4 builds scenes from tensors
 * (float vertices, integer indices, material, light and camera).  All triangles are both occluders and reflectors
 * (two-sided Lambertian, flat face normal); triangles listed in light_tris
 * also emit `radiance` from their front face (counter-clockwise winding). */
typedef struct {
  const float* verts;          /* [n_verts,3] world positions */
  int32_t n_verts;
  const int32_t* tris;         /* [n_tris,3] vertex indices */
  int32_t n_tris;
  const float* albedo;         /* [n_tris,3] Lambertian albedo (or constant colour, see primary_only) */
  const int32_t* light_tris;   /* [n_light_tris] indices into tris; may be NULL if n_light_tris == 0 */
  int32_t n_light_tris;
  const float* radiance;       /* [3] emitted radiance of every light triangle */
  const float* cam_to_world;   /* [4,4] row-major affine camera matrix; camera looks down -z, y up */
  float cam_scale;             /* pinhole: tan(fov_y/2); ortho: half height of the view; fisheye: the
                                  angle from the optical axis at half the image height (radians) */
  int32_t cam_type;            /* DRT_CAMERA_ORTHO, DRT_CAMERA_PINHOLE or DRT_CAMERA_FISHEYE */
  int32_t width, height;       /* image size in pixels */
  int32_t bvh_leaf_size;       /* most triangles per BVH leaf, 1..8 (0 selects 1).  Two suit work
                                  dominated by coherent first-vertex rays (direct lighting: 4 %
                                  faster), one suits many incoherent rays (path tracing) */
} drt_scene_desc;

/* Sampling options of one render/backward pair. */
typedef struct {
  int32_t spp;          /* interior samples per pixel (Eq. gradient_monte_carlo) */
  int32_t edge_spp;     /* primary edge samples = edge_spp * width * height, spread over the
                           screen by the edge-length CDF (Sec. 5.2.1) */
  int32_t max_depth;    /* scattering vertices per path: 1 = direct lighting; >1 path tracing */
  int32_t primary_only; /* 1: radiance = albedo of the first hit (no lighting), 0: lit */
  uint64_t seed;        /* Philox key */
  float eps_rel;        /* edge side offset: eps_rel*max(W,H) pixels for primary edges and
                           eps_rel*|omega| for secondary edges (the two-sided evaluation of
                           Sec. 5.2.1 needs a small offset); <= 0 selects 2^-16 */
  int32_t terms;        /* gradient terms: bit0 interior, bit1 primary edges, bit2 secondary
                           edges; 0 selects all */
  int32_t proposal;     /* primary edge proposal: 0 edge by clipped screen length (Sec. 5.2.1);
                           1 tile segment by q = 1/2 len/L + 1/2 w/W with the segment weights
                           below (every segment keeps q >= 1/2 len/L, so the estimator stays
                           unbiased; see drt_scene_segments for the segment list);
                           2 the same mixture with w_k = len_k exp(clamp(s_k, -40, 40)), where
                           s_k = seg_weights[k] is a network score (drt_mlp_forward), a log
                           contribution density per unit screen length */
  const float* seg_weights;  /* [n_seg_weights] device array: nonnegative weights (proposal 1) or
                                scores (proposal 2) */
  int64_t n_seg_weights;
  float* seg_log;       /* proposal 1 or 2, may be NULL: device [n_seg]; each primary edge sample
                           adds |w . (f_u - f_l)| to its segment (training data of the network) */
  int32_t scene_id;     /* >= 0: fourth word of every Philox counter.  A batch (drt_batch_*)
                           gives scene k of the batch scene_id k, so a single-scene call
                           with scene_id k reproduces it; 0 otherwise */
  int32_t sec_sampler;  /* secondary edge selection at a shading vertex: 0 by 3D edge length
                           (Sec. 5.2.2); 1 through the edge hierarchy of Sec. 5.3.1 (camera-
                           silhouette edges by 3D position, the rest by position and the Hough
                           points of their face planes; at the last vertex, v-sphere culling of
                           non-silhouettes and a light-cone bound (boxes whose directions from
                           the shading point miss the lights' bounding sphere); importance
                           length x cosine bound / distance;
                           samples split between children, one edge kept by weighted
                           reservoir sampling and weighted by its resampling weight).  The
                           hierarchy is built on the backward call's stream when the scene is
                           new or changed (device memory about 200 bytes per edge).  A batch
                           takes 0 only. */
  int32_t sec_tree_samples;  /* sec_sampler 1: samples distributed from the root, 1..64;
                                0 selects 16 */
  int32_t sec_point;    /* point on a secondary edge (Sec. 5.3.2): 0 uniform in the edge
                           parameter (Sec. 5.2.2); 1 by the clamped cosine of the shading point
                           integrated along the edge's arc (the linearly transformed cosine of
                           a Lambertian surface is the cosine itself), closed-form CDF and
                           inverse, mixed 1/4 with uniform so every point keeps a positive
                           density.  A batch takes 0 only. */
  int32_t pix_begin, pix_end;   /* backward: evaluate the interior and secondary terms only for the
                                   samples of pixels p (row-major index) with pix_begin <= p < pix_end;
                                   pix_end <= 0 selects every pixel.  With the edge range below, a
                                   full-size gradient can be checked entry by entry against a
                                   reference that evaluates the same samples one by one */
  int64_t edge_begin, edge_end; /* backward: evaluate only the primary edge samples with index j,
                                   edge_begin <= j < edge_end (the index that selects the sample's
                                   random numbers, before the samples are sorted by screen position);
                                   edge_end <= 0 selects every sample */
  int32_t aov;                  /* geometry buffers (the AOV extension of Sec. 5.4): 0 the image as set
                                   by primary_only; 1 the albedo of the first hit (same as
                                   primary_only = 1); 2 the world position of the first hit; 3 its
                                   unit shading normal, flipped to face the ray; 4 its distance from
                                   the ray origin (in all three channels).  Pixels without a hit are
                                   0.  aov > 0 implies primary_only; the backward pass returns the
                                   interior derivative of the buffer and the primary edge term of
                                   its discontinuities, so a deferred shading of the buffers written
                                   by the caller differentiates end to end */
  int32_t sec_nee;              /* 1: next-event estimation for edges (Sec. 5.3.3) beside the length
                                   sampler.  At every shading vertex the shadow ray of next-event
                                   estimation is drawn again; the edges whose billboards (width
                                   nee_width, facing the ray: the two lines pass within half the
                                   width, at an edge parameter in [0, 1], before the light point)
                                   it crosses race for one more secondary sample (key -ln U /
                                   importance; importance length / distance, zero off the silhouette
                                   seen from the vertex, at or below its tangent plane, or within
                                   the width of the vertex).  Both
                                   samples are weighed by the balance heuristic 1 / (p_length +
                                   width p_billboard) over an auxiliary offset, which keeps the term
                                   unbiased.  Needs sec_sampler 0 and sec_point 0
                                   (DRT_ERR_INVALID_ARG otherwise); builds the edge hierarchy for
                                   its crossing queries; doubles the secondary scratch.  The batch
                                   and the allocation-free backward take 0 only. */
  float nee_width;              /* sec_nee: billboard width; <= 0 selects the L2 norm over the
                                   three coordinates of 2 % of the vertices' mean absolute
                                   deviation, computed on the backward call's stream */
  int32_t spp_per_pass;         /* > 0 and < spp: the interior samples in P = spp / spp_per_pass passes
                                   (spp must be a multiple), which bounds the tape to one pass (the
                                   checkpoint of Sec. 5.4 then holds spp_per_pass paths per pixel).
                                   Pass p draws spp_per_pass samples per pixel with the Philox key
                                   seed + p * 0x9E3779B97F4A7C15 (mod 2^64); the image is the mean of
                                   the passes' images and the gradient the sum of their gradients
                                   with d_image / P.  drt_render returns the last pass's tape;
                                   drt_render_backward renders every pass again into scene-owned
                                   scratch (the tape argument may be NULL) and runs the primary edge
                                   term once with the full edge_spp and the key seed.  0: one pass.
                                   The batch and the allocation-free backward take 0 only. */
} drt_render_opts;

/* Gradient outputs: device or host arrays, each may be NULL (not wanted).
 * Values are ADDED to what the arrays hold.
 * Flat parameter layout (jac_param): [0, 3V) vertex coordinates (vertex-
 * major), [3V, 3V+3T) albedo, then radiance (3), camera rows 0..2 (12),
 * camera scale (1). */
typedef struct {
  float* d_verts;        /* [n_verts,3] */
  float* d_albedo;       /* [n_tris,3] */
  float* d_radiance;     /* [3] */
  float* d_cam_to_world; /* [3,4] rows 0..2 of the camera matrix */
  float* d_cam_scale;    /* [1] */
  float* dimage_dparam;  /* [n_jac,H,W] or NULL: per-pixel gradient image (drt_render_backward only): for
                            each listed parameter k and pixel p, the part of d loss / d theta_k that the
                            samples of pixel p contribute (interior and secondary samples by their camera
                            path's pixel, primary edge samples by the pixel containing their point; summed
                            over the pixels it is the gradient entry).  With d_image set to one pixel's
                            channel weights it is that pixel's derivative; with d_image = 1 it is the
                            derivative image of the summed channels, the per-pixel images of the
                            finite-difference validation of Sec. 5.4.1 */
  int32_t n_jac;         /* 0..8 listed parameters */
  int32_t pad_;
  int64_t jac_param[8];  /* their flat indices (layout above) */
} drt_grads;

/* Create a context on CUDA device `device` (owns the device error flag and
 * scratch pools).  out receives the handle. */
drt_status drt_create(int device, drt_context** out);
drt_status drt_destroy(drt_context* ctx);

/* Upload a scene and build everything derived from it: the LBVH over the
 * triangles (Morton codes, radix sort, Karras hierarchy, bottom-up refit), the
 * unique edge list, the light-area CDF, the CDF of projected and clipped
 * screen-space edge lengths used to pick primary edges (Sec. 5.2.1) and the
 * 3D edge-length CDF for secondary visibility.  Enqueued on stream.
 * Errors: DRT_ERR_INVALID_ARG for out-of-range indices or sizes (checked on
 * the host); non-finite vertices raise the device flag. */
drt_status drt_scene_upload(drt_context* ctx, const drt_scene_desc* desc, void* stream, drt_scene** out);

/* Replace the vertex positions (same topology) and rebuild the LBVH and the
 * edge CDFs -- one step of an optimisation loop.  verts: [n_verts,3]. */
drt_status drt_scene_update_vertices(drt_context* ctx, drt_scene* scene, const float* verts, void* stream);

/* Replace per-triangle albedo [n_tris,3] / radiance [3] / camera [4,4] and scale. */
drt_status drt_scene_update_params(drt_context* ctx, drt_scene* scene, const float* albedo, const float* radiance,
                                   const float* cam_to_world, const float* cam_scale, void* stream);
drt_status drt_scene_free(drt_context* ctx, drt_scene* scene);

/* Forward pass (Eq. first estimated by Eq. gradient_monte_carlo): image
 * [H,W,3] = per-pixel mean of spp path samples with next-event estimation at
 * every vertex.  If tape != NULL every path vertex is checkpointed (the
 * per-vertex checkpointing of Sec. 5.4) in a library-owned tape that the
 * backward pass reads (12 bytes per sample and vertex); free it with
 * drt_tape_free.  If *tape already holds a tape of this scene large enough
 * for these options it is overwritten in place (no allocation); any other
 * non-NULL *tape is freed and replaced. */
drt_status drt_render(drt_context* ctx, drt_scene* scene, const drt_render_opts* opts, float* image,
                      drt_tape** tape, void* stream);

/* Backward pass: given d_image = d loss / d image [H,W,3], ADD d loss / d
 * parameter to grads.  Interior term: hand-written reverse sweep over the
 * checkpointed path, from the last vertex back to the camera (Sec. 5.4).
 * Primary edges: Eq. mc with the edge-equation derivatives of
 * Eq. redner_dirac_jacobian, chained through the projection.  Secondary
 * edges: Eq. dirac_3d_edge at every path vertex.  tape must come from
 * drt_render on this scene with the same opts (else DRT_ERR_STATE).  tape
 * may be NULL when max_depth == 1 (the camera paths are traced again) or
 * when neither the interior nor the secondary term is asked for; otherwise
 * a NULL tape is DRT_ERR_INVALID_ARG. */
drt_status drt_render_backward(drt_context* ctx, drt_scene* scene, const drt_tape* tape,
                               const drt_render_opts* opts, const float* d_image, const drt_grads* grads,
                               void* stream);
drt_status drt_tape_free(drt_context* ctx, drt_tape* tape);

/* drt_render_backward without any memory allocation.  The paper has no
 * counterpart; this entry point exists for callers that cannot allocate
 * device memory inside their step: a loop that reserved the device memory up
 * front through its own caching allocator (a cudaMalloc there can fail, or
 * force the allocator to hand its cache back and stall), or a process held
 * to a fixed device memory budget.  Arguments and results are those of
 * drt_render_backward, except:
 *   - d_image and every non-NULL gradient array must be device memory (no
 *     host staging); otherwise DRT_ERR_INVALID_ARG.
 *   - Only the length proposal for primary edges: opts->proposal != 0 is
 *     DRT_ERR_INVALID_ARG (the mixture proposals build their CDF in
 *     scene-owned buffers that grow on demand).
 *   - No next-event estimation for edges and one sample pass: opts->sec_nee
 *     != 0 or 0 < spp_per_pass < spp is DRT_ERR_INVALID_ARG (scene-owned
 *     scratch).
 *   - With the edge hierarchy (sec_sampler 1) the hierarchy's buffers must
 *     exist from an earlier drt_render_backward with it on this scene, else
 *     DRT_ERR_STATE; a scene changed since is rebuilt in place.
 *   - The scratch (one row of 16 partial sums per thread block, plus the
 *     totals of the first reduction stage) is a fixed array of 2^22 floats
 *     (16 MiB) compiled into the library, which every GPU that loads the
 *     library holds until the process exits.  It holds about 2^18 rows: a
 *     512x512 image at 64 spp and 64 edge samples per pixel needs 98304.
 *     Larger jobs are rejected with DRT_ERR_INVALID_ARG and a message
 *     giving the sizes.
 *   - Every call made outside stream capture looks up the array's device
 *     address with cudaGetSymbolAddress (the context's device must be
 *     current); a call during capture uses the last address found, so make
 *     the first call on a device before any stream capture.
 *   - All calls share the one array, and every call overwrites the rows it
 *     reads before reading them; calls that overlap on the GPU (other streams,
 *     other threads) race on it and must be serialised by the caller. */
drt_status drt_render_backward_noalloc(drt_context* ctx, drt_scene* scene, const drt_tape* tape,
                                       const drt_render_opts* opts, const float* d_image, const drt_grads* grads,
                                       void* stream);

/* ---- Batched scenes ------------------------------------------------------
 * A batch runs render and backward of n uploaded scenes as one step (a
 * project addition: the thesis renders one scene per call).  Each pass
 * (render; interior or path; secondary edges; primary edges) is one
 * persistent launch whose CTAs take (scene, block) work items from an atomic
 * counter; the primary edge samples of all scenes are sorted by screen
 * position in one radix sort; the global gradients of each scene are reduced
 * in a fixed order.  Scene k uses scene_id k for its random numbers: its
 * image equals drt_render of that scene with opts.scene_id = k bit for bit,
 * and its gradients equal drt_render_backward's with a tape, up to the order
 * of floating-point atomic additions into vertex and albedo gradients (and,
 * after autotuning of the edge budget, the grouping of the global partial
 * sums).  A batch uses its own tapes and scratch; scenes may repeat.
 * Arrays of a batch are device memory and must outlive it. */
typedef struct {
  drt_scene* scene;
  float* image;            /* [H,W,3], written by every run */
  const float* d_image;    /* [H,W,3] d loss / d image, or NULL: no backward pass for this scene */
  drt_grads grads;         /* accumulated (+=) by every run; each array may be NULL */
  const float* verts;      /* [V,3] or NULL; if set, every run first copies these vertices into the
                              scene and rebuilds its BVH and edge tables, as
                              drt_scene_update_vertices does */
} drt_batch_item;

typedef struct {
  int32_t ctas_per_sm[5];  /* per pass (render, interior, secondary, path, primary edges):
                              resident CTAs per SM of its persistent launch (the secondary
                              pass has no items: a batch queues its secondary edge samples
                              and traces them per scene) */
  int32_t grid[5];         /* CTAs launched per pass (0: the pass does not run) */
  int32_t chunk[5];        /* work items taken per counter increment */
  int32_t edge_per_thread_mult;  /* primary edge samples per thread, over the single-scene value */
  int32_t graph;           /* 1 once the step is a captured CUDA graph */
  int32_t tuned;           /* 1 if the shapes above were chosen by timing */
  int64_t items[5];        /* work items per pass */
  int64_t edge_samples;    /* primary edge samples of all scenes */
  double tune_ms;          /* host time spent tuning */
} drt_batch_info;

/* Plan a batch of n >= 1 items with shared options (proposal must be 0;
 * scene_id is set per item).  use_graph: the first run captures the step
 * into a CUDA graph, later runs replay it.  autotune: the first run times
 * candidate launch shapes per pass (probe gradients go to scratch) and
 * synchronises the stream; the result is reused by later batches of the
 * same size class on the device.  Errors: DRT_ERR_INVALID_ARG (NULL items,
 * host arrays, proposal != 0, too many samples), DRT_ERR_OOM. */
drt_status drt_batch_create(drt_context* ctx, const drt_batch_item* items, int32_t n, const drt_render_opts* opts,
                            int32_t use_graph, int32_t autotune, drt_batch** out);
/* One step of the batch on `stream`. */
drt_status drt_batch_run(drt_context* ctx, drt_batch* batch, void* stream);
drt_status drt_batch_get_info(drt_context* ctx, const drt_batch* batch, drt_batch_info* info);
/* Waits for the device, then frees the batch's buffers and graph. */
drt_status drt_batch_free(drt_context* ctx, drt_batch* batch);
/* One-shot batch without graph or tuning: images[k] (and, if d_images is
 * non-NULL, a backward pass with d_images[k] into grads[k]) for scenes[k].
 * Synchronises the stream. */
drt_status drt_render_batch(drt_context* ctx, drt_scene* const* scenes, int32_t n, const drt_render_opts* opts,
                            float* const* images, const float* const* d_images, const drt_grads* grads,
                            void* stream);

/* ---- Learned edge proposal ------------------------------------------------
 * A 3-layer network scores screen-tile segments (drt_scene_segments); its
 * scores are the segment scores of proposal 2.  It takes
 * the role of the edge importance of Sec. 5.3.1 (hierarchy with length,
 * distance and BRDF bounds); the mixture with the length proposal keeps the
 * estimator unbiased whatever the network outputs.
 *   y = w3 . relu(W2 relu(W1 x + b1) + b2) + b3,  x in R^32, hidden width 64,
 * BF16 weights and activations (tcgen05 tensor cores), FP32 accumulation.
 * All arrays are device memory; weights are [out, in] row-major. */
typedef struct {
  const void* w1;   /* [64,32] bf16 */
  const float* b1;  /* [64] */
  const void* w2;   /* [64,64] bf16 */
  const float* b2;  /* [64] */
  const float* w3;  /* [64] */
  const float* b3;  /* [1] */
} drt_mlp_weights;
typedef struct {
  float *w1, *b1, *w2, *b2, *w3, *b3;  /* FP32 gradients, same shapes; values are ADDED */
} drt_mlp_grads;

/* y [m] = network(x [m,32] bf16). */
drt_status drt_mlp_forward(drt_context* ctx, const void* x, int64_t m, const drt_mlp_weights* w, float* y,
                           void* stream);
/* Gradient of L = inv_n/2 * sum_r mask_r (y_r - target_r)^2 added into g;
 * L added into *loss (device scalar). */
drt_status drt_mlp_backward(drt_context* ctx, const void* x, const float* target, const float* mask, int64_t m,
                            float inv_n, const drt_mlp_weights* w, drt_mlp_grads* g, float* loss, void* stream);
/* Adam with bias correction (step >= 1) on n FP32 parameters; if params_bf16
 * is non-NULL its BF16 copy is refreshed. */
drt_status drt_adam_step(drt_context* ctx, float* params, const float* grads, float* m1, float* m2, void* params_bf16,
                         int64_t n, float lr, float beta1, float beta2, float eps, int32_t step, void* stream);

/* ---- Training the network from logged edge contributions ----------------
 * The training data come from the plain sampler itself: backward passes of
 * the primary edge term with proposal 1 and all segment weights 0 (the
 * length distribution over the tile segments) add |w . (f_u - f_l)| of every
 * primary edge sample to its segment (opts.seg_log).  One drt_mlp_log holds
 * one scene's record. */
typedef struct {
  const void* x;          /* [n,32] bf16 features of the segments (drt_segment_features), device */
  const float* seg_log;   /* [n] logged sums of |w . (f_u - f_l)| per segment, device */
  const double* seg_len;  /* [n] screen lengths of the segments (drt_scene_segments), device */
  int64_t n;              /* segments (rows) */
  double n_samples;       /* primary edge samples behind seg_log (passes x edge_spp x W x H) */
} drt_mlp_log;

/* The network's parameters and optimiser state, all device arrays in the
 * order w1 [64,32], b1 [64], w2 [64,64], b2 [64], w3 [64], b3 [1]. */
typedef struct {
  float* p[6];      /* FP32 master weights, updated in place */
  float* m1[6];     /* Adam first moments */
  float* m2[6];     /* Adam second moments */
  float* g[6];      /* gradients of the last step (overwritten every step) */
  void* w1_bf16;    /* [64,32] BF16 copy of w1 read by drt_mlp_forward, refreshed every step */
  void* w2_bf16;    /* [64,64] BF16 copy of w2 */
  int64_t step;     /* Adam steps taken so far; advanced by drt_mlp_train */
} drt_mlp_state;

typedef struct {
  int32_t steps;        /* Adam steps of this call (>= 0) */
  int32_t batch;        /* rows per step; 0 selects 16384 (at most the number of rows) */
  float lr;             /* peak learning rate; 0 selects 3e-3 (cosine decay to lr/10 over the call) */
  float delta;          /* offset of the target's logarithm; 0 selects 1e-3 */
  uint64_t seed;        /* shuffle of the rows */
  float* loss;          /* device [1] or NULL: the steps' losses are added to it */
  float* rows_target;   /* device or host [rows] or NULL: the training targets in shuffled order */
  float* rows_mask;     /* device or host [rows] or NULL: the regression weights in shuffled order */
  int64_t* rows_index;  /* device [rows] or NULL: the concatenated row behind each training row */
} drt_mlp_train_opts;

/* Train the network on the rows of n_logs logged scenes (the project's
 * counterpart of the thesis's edge importance of Sec. 5.3.1, learned from the
 * plain sampler's edge contributions).  For a segment of screen length len
 * with logged sum S out of N logging samples, in a scene whose segments total
 * screen length L and logged sum S_tot, S L / N estimates the segment's
 * integral of |w . (f_u - f_l)|; the target is
 *   log( (S L / (N len)) / (S_tot / N) + delta )
 * (the log contribution density per unit length relative to the scene's
 * mean) and the regression weight len / (L / n).  The rows of all scenes are
 * concatenated in order and shuffled by sorting one Philox draw per row
 * (counter (row, 0, 0x4D4C5054, 0), key = seed); training step i uses the
 * batch (i mod floor(rows/batch)) of the shuffled rows, the loss of
 * drt_mlp_backward with inv_n = 1/batch and bias-corrected Adam (0.9, 0.999,
 * 1e-8) at lr (0.55 + 0.45 cos(pi i / steps)).  Allocates its scratch,
 * synchronises `stream` before returning.  Errors: DRT_ERR_INVALID_ARG (NULL
 * arrays, host log arrays, empty logs, more than 2^31 - 1 rows), DRT_ERR_OOM,
 * DRT_ERR_CUDA, DRT_ERR_TIMEOUT-class device flags through drt_check_device. */
drt_status drt_mlp_train(drt_context* ctx, const drt_mlp_log* logs, int32_t n_logs, const drt_mlp_train_opts* o,
                         drt_mlp_state* state, void* stream);

/* Features of every tile segment for the network, [n_seg, 32] bf16 device
 * array (n_seg from drt_scene_segments): tile centre, segment end points,
 * lengths, camera-space normals of the edge's faces, silhouette and boundary
 * flags, albedo difference, light flag, inverse depth, edge direction, the
 * mean |d_image| of the segment's tile (d_image [H,W,3] device), and camera
 * rays traced at the segment midpoint (one through it, one half a pixel to
 * each side of the edge): whether the edge is visible there, whether the two
 * sides see different triangles or only one sees the background, the albedo
 * difference of what they see and whether one sees a light; the mean
 * |d_image| at four points along the segment over the image mean; and, if
 * image ([H,W,3] device, the rendered image of the step; may be NULL) is
 * given, the radiance contrast across the edge read from it 1.5 pixels to
 * each side of the segment midpoint, relative and log-compressed (zero
 * without an image). */
drt_status drt_segment_features(drt_context* ctx, drt_scene* scene, const float* d_image, const float* image, void* x,
                                void* stream);

/* Screen-tile segments of the clipped primary edges: every clipped edge is
 * cut where it crosses the 16-pixel tile grid (FP32 crossing parameters in
 * increasing order).  Builds them for the scene's current state (this call
 * synchronises `stream`), stores *n, and if the arrays are non-NULL writes
 * up to cap entries: edge_tile [cap,2] int32 (edge index in the sorted unique
 * edge list, tile index row-major), s01 [cap,2] float32 (edge parameters),
 * lens [cap] float64 (screen lengths).  Arrays may be host or device memory.
 * The learned proposal scores these segments (proposal 1 of drt_render_opts). */
drt_status drt_scene_segments(drt_context* ctx, drt_scene* scene, int64_t* n, int32_t* edge_tile, float* s01,
                              double* lens, int64_t cap, void* stream);

/* Closest-hit query through the scene's LBVH for n rays (test and debug
 * entry point; the render kernels use the same traversal).  o, d: [n,3]
 * origins and directions; tri: [n] hit triangle or -1; tb1b2: [n,3] =
 * (t, b1, b2).  Hits have t > 0, ties on t go to the lowest triangle id
 * (Sec. 5.2.1 relies on exact visibility; see the watertight test of Woop et
 * al. 2013 used for every ray). */
drt_status drt_debug_closest(drt_context* ctx, drt_scene* scene, int64_t n, const float* o, const float* d,
                             int32_t* tri, float* tb1b2, void* stream);

/* Profiling (off by default).  When enabled, every kernel launch of the
 * library is bracketed by CUDA events recorded on its stream; drt_profile_read
 * synchronises on them and returns, per kernel name (first-launch order), the
 * summed device time in ms and the launch count, then clears the record.
 * names: [max][64] chars (may be NULL); ms, launches: [max]; *n: entries. */
drt_status drt_profile_enable(drt_context* ctx, int enable);
drt_status drt_profile_read(drt_context* ctx, int max, char* names, double* ms, int64_t* launches, int* n);

/* Work counters (off by default): per kernel slot (0 render (the first vertex
 * of its paths beyond depth 1), 1 backward interior, 2 backward primary edges
 * (the first vertex of their side paths beyond depth 1), 3 debug, 4 backward
 * secondary edges in one kernel (depth 1), 5 and 6 the side-ray and
 * continuation stages of the secondary edges beyond depth 1, 7 the
 * continuation stages of the primary edges, 8 the continuation stages of the
 * render) four int64 counts -- rays traced to the closest hit, shadow rays,
 * BVH nodes visited, triangle tests.  drt_counters_read synchronises the
 * device, copies [9][4] counts to out and resets them. */
drt_status drt_counters_enable(drt_context* ctx, int enable);
drt_status drt_counters_read(drt_context* ctx, int64_t* out);

/* Peak probes: measurement aids for the rooflines of the ray kernels (not
 * part of the method; the paper has no counterpart).  Both allocate a small
 * device buffer, run on `stream`, synchronise it and return the best of five
 * event-timed launches.
 * drt_probe_fma: FP32 lane-operations per second of a kernel running eight
 *   independent FMA chains per thread at 2048 threads per SM (each FMA
 *   counts as one lane-operation).
 * drt_probe_l2: bytes per second (read + write) of a copy between two
 *   buffers of bytes/2 each, 64 passes per launch, loads and stores cached
 *   in L2 only; bytes in [1 MiB, 1 GiB] (choose it well below the L2 size to
 *   measure L2).  Errors: DRT_ERR_INVALID_ARG, DRT_ERR_OOM, DRT_ERR_CUDA. */
drt_status drt_probe_fma(drt_context* ctx, double* lane_ops_per_s, void* stream);
drt_status drt_probe_l2(drt_context* ctx, int64_t bytes, double* bytes_per_s, void* stream);

/* Synchronise stream and read the device error flag: DRT_OK, or
 * DRT_ERR_DEVICE_FLAG with *code / *info (may be NULL) set and the flag
 * cleared. */
drt_status drt_check_device(drt_context* ctx, void* stream, int32_t* code, int32_t* info);

/* Message of the last failing call on this thread (thread-local storage,
 * valid until the next failing call on the thread).  ctx may be NULL: the
 * message is kept per thread, so a failure before a context exists (e.g. in
 * drt_create) is reported too. */
const char* drt_last_error(drt_context* ctx);

/* Library version string. */
const char* drt_version(void);

#ifdef __cplusplus
}
#endif
#endif /* DRT_H */
