/*
 * ges.h -- C ABI of libges, a GB300 (sm_103a) rasterizer for Generalized
 * Exponential Splatting (Hamdi et al., "GES: Generalized Exponential Splatting
 * for Efficient Radiance Field Rendering").
 *
 * The library renders a set of 3D primitives, each with mean mu, scale s,
 * rotation quaternion q, shape parameter beta, opacity kappa and spherical
 * harmonic (SH) colour coefficients (Sec. 4.1), to an image: projection of the
 * beta-modified covariance to a 2D conic (Sec. 4.1, EWA; Sec. 4.2, Eq. approx),
 * tile|depth keys and a radix sort, front-to-back compositing with the GEF
 * falloff exp(-1/2 q^(beta/2)) (Sec. 4.1, Eq. ges; Sec. 4.2, Eq. transmittance),
 * and the gradients of all primitive parameters (backward pass).
 *
 * Conventions shared by every entry point
 *  - All functions are extern "C", never throw, and return ges_status.
 *    On failure ges_last_error() returns a message for the calling thread.
 *  - "stream" is a cudaStream_t passed as void* (NULL = legacy default stream).
 *    Work is stream-ordered: a call returns once its kernels are enqueued,
 *    unless its comment says it synchronises.
 *  - Array arguments are caller-owned DEVICE pointers to contiguous fp32 (or
 *    the stated type), row-major, unless stated otherwise.  Workspaces
 *    (ges_ctx, ges_frame, ges_server) are library-owned.
 *  - Parameters are physical values: scale > 0, opacity in (0,1), beta > 0.
 *    (The paper trains beta shifted by -2 and scale/opacity through log/logit
 *    activations, App. B.2; that reparameterisation is the caller's.)
 *    Primitives with a non-finite or non-positive beta, a zero quaternion,
 *    opacity <= alpha_min, depth <= znear, or a footprint off the image are
 *    culled (contribute nothing, receive zero gradient).
 *  - Quaternions are (w,x,y,z) and are normalised inside; their gradient is
 *    with respect to the unnormalised input.
 *  - Camera: OpenCV axes (+x right, +y down, +z forward); viewmat maps world
 *    to camera; pixel (i,j) is sampled at (i+0.5, j+0.5).
 *  - Images are planar [3, H, W]; per-pixel arrays are [H, W].
 */
#ifndef GES_H
#define GES_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum ges_status {
  GES_OK = 0,
  GES_ERR_INVALID_ARG = 1,  /* a pointer, size or value is out of range; nothing was enqueued */
  GES_ERR_OOM = 2,          /* a device allocation failed or the HBM budget would be exceeded */
  GES_ERR_CUDA = 3,         /* a CUDA runtime call failed (message names it) */
  GES_ERR_CAPACITY = 4,     /* the duplicate-key count exceeded the frame's key capacity */
  GES_ERR_NOT_READY = 5,    /* serving: the request has not finished */
  GES_ERR_TIMEOUT = 6,      /* serving: the wait ran out */
  GES_ERR_BUSY = 7,         /* serving: the request queue is full */
  GES_ERR_DEVICE_WAIT = 8   /* a bounded device-side wait gave up (status word set by a kernel) */
} ges_status;

typedef enum ges_falloff {
  /* exp(-1/2 q^(beta/2)) on the phi_bar-scaled covariance (Eq. ges with Eq. approx); default */
  GES_FALLOFF_GEF = 0,
  /* exp(-1/2 q) on the phi_bar-scaled covariance: the paper's Gaussian-form
     rasterizer that only rescales the splat (Sec. 4.2, "Approximate Rasterization") */
  GES_FALLOFF_PAPER_APPROX = 1
} ges_falloff;

typedef enum ges_phi_mode {
  /* phi_bar_rho(beta) = 2 / (1 + exp(-(rho beta - 2 rho))) on the scale vector (Eq. approx); default */
  GES_PHI_APPROX = 0,
  /* the exact Gamma ratio of Eq. probablity normalised to 1 at beta = 2,
     phi_n(beta) = 2 Gamma(3/beta) / Gamma(1/beta), on the scale vector (the slot phi_bar approximates).
     phi_n is 4 at beta = 1, 240 at beta = 1/2 and over 1e5 below beta = 0.33: primitives of small beta
     grow accordingly (the instability Sec. 4.2 gives as the reason for phi_bar) */
  GES_PHI_EXACT = 1,
  /* phi_n read as a ratio of variances (Eq. effective): sqrt(phi_n(beta)) on the scale vector */
  GES_PHI_EXACT_VARIANCE = 2
} ges_phi_mode;

typedef struct ges_camera {
  int32_t width, height;  /* pixels, 1..16384 each */
  float fx, fy, cx, cy;   /* pinhole intrinsics in pixels */
  float viewmat[16];      /* world -> camera, row-major 4x4 (last row 0,0,0,1) */
  float campos[3];        /* camera centre in world space (SH view direction) */
  float znear;            /* primitives with camera depth <= znear are culled */
  float bg[3];            /* background colour composited with the final transmittance */
} ges_camera;

typedef struct ges_params {
  float rho;              /* shape strength of phi_bar (App. B.2: 0.1) */
  int32_t falloff;        /* ges_falloff */
  float dilation;         /* added to the 2D covariance diagonal, px^2 (0.3) */
  float alpha_max;        /* alpha clamp (0.99) */
  float alpha_min;        /* fragments with alpha below this are skipped (1/255) */
  float t_min;            /* stop before transmittance would drop below this (1e-4) */
  float extent_margin_rel;/* relative safety margin on the tile extent (1e-3) */
  float extent_margin_abs;/* absolute safety margin on the tile extent, px (1e-2) */
  float clamp_fov;        /* tangent clamp of the EWA Jacobian, in half-image units (1.3) */
  int32_t segment_tiles;  /* binning granularity: tiles per list segment along x, a power of two
                             in [1, 1024] (16).  Each tile row is cut into segments of this many
                             tiles and a primitive is listed once per segment its extent meets
                             (1 lists every tile separately).  Larger segments mean fewer entries
                             to sort and more entries for the composite to skip; the images do
                             not depend on it. */
  int32_t phi_mode;       /* ges_phi_mode: the scale modification (GES_PHI_APPROX).  rho is used by
                             GES_PHI_APPROX only.  The exact forms take ln Gamma on the key path's
                             fixed-order FP32 arithmetic (Stirling's series after a shift to >= 4),
                             so their phi is within 2e-6 of the exact ratio for beta in [0.4, 32] */
} ges_params;

typedef struct ges_scene {
  int64_t n;              /* number of primitives, 0..2^31-1 */
  int32_t sh_degree;      /* 0..3 */
  const float* means;     /* [n,3] */
  const float* scales;    /* [n,3], > 0 */
  const float* quats;     /* [n,4] (w,x,y,z) */
  const float* betas;     /* [n], > 0 */
  const float* opacities; /* [n], in (0,1) */
  const float* shs;       /* [n,(sh_degree+1)^2,3], l-major, m = -l..l, real SH with Condon-Shortley phase */
} ges_scene;

typedef struct ges_grads { /* same shapes as ges_scene; written (not accumulated) by ges_render_bwd */
  float* means;
  float* scales;
  float* quats;
  float* betas;
  float* opacities;
  float* shs;
} ges_grads;

typedef struct ges_ctx ges_ctx;
typedef struct ges_frame ges_frame;
typedef struct ges_server ges_server;

/* Message for the last failed call on this thread ("" if none).  Owned by the library. */
const char* ges_last_error(void);

/* Defaults listed beside each ges_params field. */
ges_status ges_params_default(ges_params* out);

/* Library context on CUDA device `device`.  hbm_budget_bytes bounds the memory this
   context may allocate (0 = no bound).  Destroy with ges_ctx_destroy. */
ges_status ges_ctx_create(int device, size_t hbm_budget_bytes, ges_ctx** out);
void ges_ctx_destroy(ges_ctx* ctx);

/* Per-frame workspace for up to n_capacity primitives at width x height.
   key_capacity: maximum number of (segment, primitive) entries K (see ges_bin_sort).  0 selects
   automatic growth: ges_bin_sort then synchronises the stream once per call to read
   K and reallocates when needed.  With key_capacity > 0 ges_bin_sort never
   synchronises (the sequence is graph-capturable); when K exceeds it the frame is
   marked overflowed, no keys are written, and ges_frame_status reports
   GES_ERR_CAPACITY.  Destroy with ges_frame_destroy (synchronises the device). */
ges_status ges_frame_create(ges_ctx* ctx, int64_t n_capacity, int32_t width, int32_t height,
                            int64_t key_capacity, ges_frame** out);
void ges_frame_destroy(ges_frame* frame);

/* Preprocess (per primitive): scale modification phi_bar (Eq. approx), covariance from
   scale and quaternion (Sec. 4.1), EWA projection to a 2D conic (Sec. 4.1), opacity-aware
   beta-dependent tile extent, depth key, SH colour.  scene->n <= n_capacity; the camera's
   size must equal the frame's.  The scene arrays must stay valid until ges_render_bwd
   (if used) has been enqueued. */
ges_status ges_preprocess(ges_frame* frame, const ges_scene* scene, const ges_camera* cam,
                          const ges_params* params, void* stream);

/* Binning: depth sort of the primitives (radix, 32-bit float keys); per primitive and tile row,
   the columns its elliptical extent spans; an exclusive scan of the entries each primitive makes
   (one per segment of params->segment_tiles tiles that its spans meet); entry generation in
   depth order; a stable radix sort by segment id; per-segment [start,end) ranges.  An entry
   carries the columns of its span inside the segment, so a tile's list (the entries of its
   segment whose span contains the tile, in order) equals a stable sort of the 64-bit keys
   (tile << 32 | depth bits) with values = primitive index, restricted to that tile.
   The depth sort runs in one sweep with a bounded decoupled look-back; should a wait ever give
   up, ges_frame_status reports GES_ERR_DEVICE_WAIT and the lists must not be used.
   With a fixed key_capacity, ges_preprocess, ges_bin_sort, ges_render_fwd and ges_render_bwd
   enqueue work only (no host synchronisation, no allocation), so one frame's sequence can be
   captured into a CUDA graph and replayed; the camera, parameters and array pointers of the
   calls are fixed in the graph. */
ges_status ges_bin_sort(ges_frame* frame, void* stream);

/* Forward composite (Sec. 4.2): per pixel, front to back over its tile's list,
   q = d^T conic d, G = exp(-1/2 q^(beta/2)) (or exp(-1/2 q)), alpha = min(alpha_max, kappa G),
   skip alpha < alpha_min, stop before T drops below t_min.  Outputs (device, caller-owned):
   img [3,H,W] = colour + T * bg, final_T [H,W], n_contrib [H,W] (1-based position, in the
   list of the tile's segment, of the last entry composited; 0 if none). */
ges_status ges_render_fwd(ges_frame* frame, float* img, float* final_T, uint32_t* n_contrib, void* stream);

/* Backward: gradients of L with respect to every scene parameter, given dL/dimg [3,H,W].
   Recomputes back to front from final_T and n_contrib as returned by ges_render_fwd for
   the same frame (no per-fragment state is stored), then chains through the projection.
   `scene` must be the one passed to ges_preprocess.  All of out's arrays are overwritten. */
ges_status ges_render_bwd(ges_frame* frame, const ges_scene* scene, const float* final_T,
                          const uint32_t* n_contrib, const float* dL_dimg, const ges_grads* out,
                          void* stream);

/* Synchronises `stream` and reports GES_ERR_CAPACITY if the last ges_bin_sort overflowed,
   else GES_OK.  *num_keys (optional) receives K, the number of (segment, primitive) entries. */
ges_status ges_frame_status(ges_frame* frame, void* stream, int64_t* num_keys);

/* Inspection (tests, tools).  Synchronises `stream`.  Expands the segment lists of the last
   ges_bin_sort into per-tile lists and copies to HOST buffers the sorted 64-bit keys
   (tile << 32 | depth bits) and values (primitive index), max_keys entries at most;
   *num_keys receives the number of (tile, primitive) entries. */
ges_status ges_frame_keys(ges_frame* frame, void* stream, uint64_t* keys, uint32_t* vals,
                          int64_t max_keys, int64_t* num_keys);

/* Inspection.  Synchronises `stream`.  Copies per-primitive results of the last
   ges_preprocess to HOST buffers (any may be NULL): depth_key [n] (float bits of the camera
   depth, 0xFFFFFFFF if culled), rect [n,4] int32 (x0,y0,x1,y1 tiles, end-exclusive),
   record [n,12] fp32 (mean x, mean y, q limit, beta exponent, conic a, b, c, opacity,
   r, g, b, 0), tile ranges [tiles,2] uint32 (into the expanded list of ges_frame_keys; empty
   tiles hold [0,0]).  Also the intermediate 2D gradients of the
   last ges_render_bwd, grad2d [n,12] (mx, my, conic a, b, c, opacity, beta exponent, r, g, b). */
ges_status ges_frame_inspect(ges_frame* frame, void* stream, uint32_t* depth_key, int32_t* rect,
                             float* record, uint32_t* ranges, float* grad2d);

/* Inspection.  Re-runs the forward composite of the last ges_bin_sort into internal scratch
   buffers while counting work, then synchronises `stream`: *evaluated receives the number of
   (fragment, pixel) pairs tested before each pixel stopped, *in_extent those whose q was within
   the primitive's extent (the pairs that evaluate the falloff), *composited those that were
   composited (alpha >= alpha_min), *num_keys K (segment entries).  Any output pointer may be
   NULL. */
ges_status ges_frame_count_work(ges_frame* frame, void* stream, int64_t* evaluated, int64_t* in_extent,
                                int64_t* composited, int64_t* num_keys);

/* Number of CUDA kernels this process has launched through libges (all threads). */
uint64_t ges_kernel_launches(void);

/* Kernel tracing (a measurement aid; no counterpart in the paper).  While tracing is on, every
   kernel launch or launch group that the frame calls of this context make (ges_preprocess,
   ges_bin_sort, ges_render_fwd, ges_render_bwd) is bracketed by two CUDA events recorded on the
   caller's stream.  The names are the kernel names, or for a group its stage:
   "k_preprocess", "depth_sort", "scan_touched", "k_keygen", "list_sort", "k_ranges",
   "k_render_fwd", "tile_order", "k_render_bwd", "k_preprocess_bwd".
   ges_trace_enable(ctx, 1) starts a new record (0 stops recording and keeps the record).
   ges_trace_read synchronises with the recorded events and writes, per name in first-launch
   order, at most `capacity` entries: names[32*i..] (NUL-terminated), launches[i], total_ms[i]
   (the summed device time).  *n_out receives the number of distinct names.  The record is then
   cleared.  Errors: GES_ERR_INVALID_ARG for a NULL ctx/n_out or capacity < 0 with non-NULL
   outputs; GES_ERR_CUDA if an event fails.  Host cost: two event records per launch. */
ges_status ges_trace_enable(ges_ctx* ctx, int on);
ges_status ges_trace_read(ges_ctx* ctx, int32_t capacity, char* names, int64_t* launches, double* total_ms,
                          int32_t* n_out);

/* Training image loss (Sec. 4.3, Eq. mask, Eq. laplace, Eq. final; no rasterizer state).

   ges_freq_mask: the frequency-modulated mask M_omega of a ground-truth image gt [3,H,W] (fp32,
   device): the channel mean of gt, box-downsampled by f = round(1/scale) (the image-frequency
   scale, 0.2), filtered by DoG_omega = G(., 0.2 + 20 omega) - G(., 0.1 + 10 omega) (separable
   Gaussian blurs truncated at ceil(3 sigma), zero outside the image); |DoG| divided by its maximum
   and compared with `threshold` (0.5); upsampled by nearest neighbour into mask [H,W] (uint8 0/1,
   device, caller-owned).  For omega <= 1/2 the mask is 1 - M_(1 - omega).  omega in [0,1] (the
   training schedule uses iteration / total iterations), scale in (0,1].

   ges_image_loss: L = (1 - lambda_ssim - lambda_omega) L1 + lambda_ssim (1 - SSIM)
   + lambda_omega L_omega (paper: 0.2 and 0.5), L1 = mean |I - I_gt|,
   L_omega = mean |(I - I_gt) M| (means over the 3 H W values; M from ges_freq_mask), SSIM with
   an 11 x 11 Gaussian window (sigma 1.5), zero padding, C1 = 0.01^2, C2 = 0.03^2.  Writes
   loss[4] = (L, L1, SSIM, L_omega) and dL_dimg [3,H,W] = dL/dI (the upstream gradient of
   ges_render_bwd); all device pointers, caller-owned; I and I_gt [3,H,W] fp32.

   Both are stream-ordered and asynchronous.  Each keeps grow-only scratch in the context (one
   buffer per call kind), so calls of one kind on one context must be ordered on one stream.
   Errors: GES_ERR_INVALID_ARG for NULL pointers, sizes or parameters out of range (nothing
   enqueued); GES_ERR_OOM if the scratch cannot be allocated. */
ges_status ges_freq_mask(ges_ctx* ctx, const float* gt, int32_t width, int32_t height, float omega, float scale,
                         float threshold, uint8_t* mask, void* stream);
ges_status ges_image_loss(ges_ctx* ctx, const float* img, const float* gt, const uint8_t* mask, int32_t width,
                          int32_t height, float lambda_ssim, float lambda_omega, float* loss, float* dL_dimg,
                          void* stream);

/* Training-side updates (Sec. 4.4; App. B.2): the optimizer and the density control that consume
   ges_render_bwd's gradients, as in Gaussian splatting (whose optimisation the paper keeps) plus
   the paper's shape resets and shape pruning.

   The optimizer's variables of a primitive, in six groups (index: contents, activation):
     0 means [n,3]                    mu = p
     1 log-scales [n,3]               s = exp(p)
     2 quaternions [n,4]              q = p (the rasterizer normalises; its gradient is w.r.t. p)
     3 shifted shapes [n]             beta = p + 2 (App. B.2: the shape is stored shifted by -2)
     4 opacity logits [n]             kappa = 1 / (1 + exp(-p))
     5 SH coefficients [n,(d+1)^2,3]  identity
   A ges_train_set holds the variables and their Adam moments (device fp32 arrays of those shapes,
   caller-owned; moments zero-initialised by the caller).  Each pointer must be 16-byte aligned. */
typedef struct ges_train_set {
  int64_t n;              /* primitives (rows); for an output set, the capacity */
  int32_t sh_degree;      /* 0..3 */
  float* param[6];
  float* m[6];            /* Adam first moments */
  float* v[6];            /* Adam second moments */
} ges_train_set;

/* Physical values written for the renderer (same shapes as ges_scene; device, caller-owned). */
typedef struct ges_scene_out {
  float* means;
  float* scales;
  float* quats;
  float* betas;
  float* opacities;
  float* shs;
} ges_scene_out;

typedef struct ges_adam_params {
  float lr[6];            /* per group; lr[5] is the SH DC rate.  App. B.2: 1.6e-4 (the position
                             schedule's start, see ges_position_lr), 0.005, 0.001, 0.001, 0.05, 0.0025 */
  float lr_sh_rest;       /* the SH coefficients of degree >= 1 (0.0025 / 20, as in Gaussian splatting) */
  float beta1, beta2;     /* 0.9, 0.999 */
  float eps;              /* 1e-15 */
} ges_adam_params;

typedef struct ges_density_params {
  float grad_threshold;   /* densify where the mean screen-space gradient norm >= this (App. B.2: 0.0003) */
  float percent_dense;    /* clone if max scale <= percent_dense * scene_extent, else split (0.01) */
  float scene_extent;     /* world units, > 0 (1) */
  float min_opacity;      /* prune kappa below this (App. B.2: 0.005); 0 disables */
  float min_beta;         /* shape pruning: prune beta below this; 0 disables (0) */
  float max_world_size;   /* prune where max scale > max_world_size * scene_extent; 0 disables (0) */
} ges_density_params;

ges_status ges_adam_params_default(ges_adam_params* out);
ges_status ges_density_params_default(ges_density_params* out);

/* The position learning rate at `step` (host only): log-linear from lr_init to lr_final over
   max_steps (constant after), times delay_mult + (1 - delay_mult) sin(pi/2 min(step/delay_steps, 1))
   when delay_steps > 0.  App. B.2: 1.6e-4, 1.6e-6, 0.01, 30000.  Errors: GES_ERR_INVALID_ARG for a
   NULL out, max_steps < 1, or a rate <= 0. */
ges_status ges_position_lr(int64_t step, float lr_init, float lr_final, float delay_mult, int64_t delay_steps,
                           int64_t max_steps, float* out);

/* One fused Adam step (Kingma & Ba, with bias correction; step >= 1 counts the calls) over every
   group: the gradient w.r.t. the physical value (grads, as ges_render_bwd writes it) is taken to
   the variable through its activation, the moments and the variable are updated, and the new
   physical values are written to phys.  One launch, one pass over the arrays.  Stream-ordered.
   Errors: GES_ERR_INVALID_ARG for NULL or misaligned pointers, n < 0, step < 1 or
   beta1/beta2 outside [0,1). */
ges_status ges_adam_step(ges_ctx* ctx, const ges_train_set* set, const ges_grads* grads, const ges_scene_out* phys,
                         const ges_adam_params* hp, int64_t step, void* stream);

/* phys = the activations of set's variables (after ges_density_control or a reset).  Stream-ordered. */
ges_status ges_activate(ges_ctx* ctx, const ges_train_set* set, const ges_scene_out* phys, void* stream);

/* Densification statistics of the frame's last ges_render_bwd: for every primitive the view lists,
   grad_accum[i] += ||(dL/du W/2, dL/dv H/2)|| (the screen-space mean gradient in NDC units, as in
   Gaussian splatting) and count[i] += 1.  grad_accum [n] fp32 and count [n] int32 (device,
   caller-owned, zeroed by the caller before the first view).  Stream-ordered.  Errors:
   GES_ERR_INVALID_ARG for NULL pointers or no ges_render_bwd since the last ges_preprocess. */
ges_status ges_densify_stats(ges_frame* frame, float* grad_accum, int32_t* count, void* stream);

/* Density control.  With g = grad_accum / max(count, 1) per row of `in`:
     clone  g >= grad_threshold and max scale <= percent_dense * extent: the row is kept and copied;
     split  g >= grad_threshold and max scale > percent_dense * extent: the row is replaced by two
            children at mu + R(q) (s * xi[i, j]) (j = 0, 1) with scales s / 1.6, the rest copied;
     prune  kappa < min_opacity, beta < min_beta, or max scale > max_world_size * extent, applied to
            every resulting row (children with their own scales).
   The decisions compare the variables with the thresholds mapped into them (log, logit, minus 2;
   computed in double on the host, rounded once to fp32).  xi: [n,2,3] fp32 standard normals
   (device), drawn by the caller.  `out` (capacity out->n rows, sh_degree as `in`, no array shared
   with `in`) receives the kept rows in order, then the clones, then the first and the second
   children, each in the order of `in`; moments are copied for kept rows and zero for new ones.
   *n_out (host) gets the row count.  The call synchronises `stream` once (to read the counts).
   Errors: GES_ERR_INVALID_ARG for NULL/misaligned pointers or parameters out of range;
   GES_ERR_CAPACITY (nothing written, *n_out = the rows needed) if out->n is too small. */
ges_status ges_density_control(ges_ctx* ctx, const ges_train_set* in, const float* grad_accum, const int32_t* count,
                               const float* xi, const ges_density_params* dp, const ges_train_set* out,
                               int64_t* n_out, void* stream);

/* Opacity reset: kappa <- min(kappa, max_opacity) (Gaussian splatting: 0.01, every 3000 steps);
   shape reset: beta <- beta (2: back to the Gaussian, every 1000 steps).  The group's moments are
   zeroed.  Stream-ordered.  Errors: GES_ERR_INVALID_ARG for NULL pointers, max_opacity outside (0,1)
   or beta <= 0. */
ges_status ges_reset_opacity(ges_ctx* ctx, const ges_train_set* set, float max_opacity, void* stream);
ges_status ges_reset_shape(ges_ctx* ctx, const ges_train_set* set, float beta, void* stream);

/* The 1D mixture-fitting study (Sec. 3.2; App. A), batched: many independent fits of one model
   with N components to 1D signals by full-batch Adam on the mean squared error.

   Models (App. A; eps = mix_eps, per component i):
     GES_MIX_GAUSSIAN  w exp(-(x - mu)^2 / (2 s^2 + eps))
     GES_MIX_DOG       w [exp(-(x - mu)^2 / (2 s^2 + eps)) - exp(-(x - mu)^2 / (2 s^2 / nu + eps))]
     GES_MIX_LOG       w (1 - (x - mu)^2 / s^2) exp(-(x - mu)^2 / (2 s^2 + eps))
     GES_MIX_GEF       w exp(-|x - mu|^beta / (2 s^2 + eps))   (beta learnt per component)
   Parameters of a run: [rows][N] with rows omega, mu, s (and beta for the GEF); w = |omega| when
   positive_weights, else omega.  Signals (App. A, width s_w, zero outside (-s_w/2, s_w/2) except
   the Gaussian): square 1, triangle s_w/2 - |x|, parabolic (s_w/2)^2 - x^2,
   half sinusoid sin((x + s_w/2) pi / s_w), exponential exp(-|x|), Gaussian exp(-x^2 / (2 s_w^2)). */
typedef enum ges_mix_model { GES_MIX_GAUSSIAN = 0, GES_MIX_DOG = 1, GES_MIX_LOG = 2, GES_MIX_GEF = 3 } ges_mix_model;
typedef enum ges_signal_kind {
  GES_SIGNAL_SQUARE = 0, GES_SIGNAL_TRIANGLE = 1, GES_SIGNAL_PARABOLIC = 2, GES_SIGNAL_HALF_SINUSOID = 3,
  GES_SIGNAL_EXPONENTIAL = 4, GES_SIGNAL_GAUSSIAN = 5
} ges_signal_kind;

typedef struct ges_fit1d_params {
  int32_t model;            /* ges_mix_model (GEF) */
  int32_t n_components;     /* N, 1..128 (5) */
  int32_t positive_weights; /* 1 (1) */
  int32_t epochs;           /* Adam steps, >= 0 (1000) */
  int32_t precision;        /* arithmetic and array element type: 32 (float) or 64 (double) (32) */
  double lr, beta1, beta2, adam_eps;  /* Adam (0.01, 0.9, 0.999, 1e-8) */
  double nu;                /* DoG variance ratio (4) */
  double mix_eps;           /* the models' eps (1e-8) */
} ges_fit1d_params;

ges_status ges_fit1d_params_default(ges_fit1d_params* out);

/* x[i] = x0 + (x1 - x0) i / (n_points - 1) and y[i] = the signal at x[i] (device arrays of the
   given precision, caller-owned).  Stream-ordered.  Errors: GES_ERR_INVALID_ARG for NULL
   pointers, an unknown kind, n_points < 1, width <= 0 or a precision other than 32/64. */
ges_status ges_signal1d(ges_ctx* ctx, int32_t kind, double width, int32_t n_points, double x0, double x1,
                        int32_t precision, void* x, void* y, void* stream);

/* `runs` fits in one launch (one CTA each).  x [n_points] (n_points <= 4096) is shared; run r fits
   y + r * y_stride (y_stride 0: one target for all).  params [runs][rows][N] holds the initial
   parameters and receives the final ones; loss_hist [runs][epochs + 1] (optional) the MSE before
   each step and after the last; final_loss [runs] the MSE after the last step; grad
   [runs][rows][N] (optional) the MSE's gradient at the final parameters.  A run whose loss stops
   being finite ends there: its later losses, its parameters and its gradient are NaN (the
   study's unstable runs).  All arrays on the device in the chosen precision.  Stream-ordered; the
   call keeps no state, so calls may run concurrently on several streams.  Errors:
   GES_ERR_INVALID_ARG for NULL pointers or parameters out of range. */
ges_status ges_fit1d(ges_ctx* ctx, const ges_fit1d_params* p, int32_t runs, int32_t n_points, const void* x,
                     const void* y, int64_t y_stride, void* params, void* loss_hist, void* final_loss, void* grad,
                     void* stream);

/* Forward render that allocates no device memory (no counterpart in the paper; it exists for
   callers that cannot allocate).  Some callers cannot call cudaMalloc: code running under another
   runtime's memory manager that has already reserved the device's memory for its own pool, or
   latency-critical loops where cudaMalloc/cudaFree are ruled out because they may synchronise the
   device.  This call computes what ges_preprocess + ges_bin_sort + ges_render_fwd compute, in the
   same kernels, for scenes of at most 65,536 primitives, images of at most 16,384 tiles (16x16
   pixels each, e.g. 2048x2048) and at most 1,048,576 (tile, primitive) duplicates.
   Arguments: scene (device arrays, as for ges_preprocess), cam, params; outputs img [3,H,W],
   final_T [H,W], n_contrib [H,W] (device, caller-owned); stream as everywhere.
   Errors: GES_ERR_INVALID_ARG for a NULL pointer or a scene/image above the limits (nothing
   enqueued); GES_ERR_CAPACITY when the duplicates exceed their limit (outputs then hold the
   background only); GES_ERR_DEVICE_WAIT when a radix sort's bounded wait on its predecessors
   gave up (outputs then undefined; a later call starts afresh); GES_ERR_CUDA for a failed launch
   or copy.  The call synchronises `stream` before returning, to read that count.
   Every intermediate buffer lives in one fixed array of about 24 MB in device global memory,
   which each GPU that loads the library holds until the process exits.  All calls share that
   array and it keeps the last call's contents: calls whose work overlaps on the GPU (other
   streams, other host threads on the same device) race on it and must be serialised by the
   caller.  The first call on each device resolves the array's address and uploads constants;
   make that first call before any stream capture on that device. */
ges_status ges_render_fwd_noalloc(const ges_scene* scene, const ges_camera* cam, const ges_params* params,
                                  float* img, float* final_T, uint32_t* n_contrib, void* stream);

/* ---------------------------------------------------------------------------------------
 * Serving: several scenes resident on the device, render requests of mixed resolutions
 * admitted by memory and batched into shared launches (continuous batching).
 * --------------------------------------------------------------------------------------- */

/* max_slots: requests that may be in flight on the device at once (1..64).
   The server runs a scheduler thread; destroy with ges_serve_destroy. */
ges_status ges_serve_create(ges_ctx* ctx, const ges_params* params, int32_t max_slots, ges_server** out);

/* Copies a scene (HOST arrays) into library-owned device memory. */
ges_status ges_serve_add_scene(ges_server* srv, const ges_scene* host_scene, int32_t* scene_id);

/* Enqueues one render; never blocks.  out_img is a HOST buffer [3,H,W] that stays valid
   until ges_serve_poll reports GES_OK for the ticket.  GES_ERR_BUSY if the queue is full. */
ges_status ges_serve_submit(ges_server* srv, int32_t scene_id, const ges_camera* cam, float* out_img,
                            uint64_t* ticket);

/* Waits up to timeout_us (0 = just check) for a ticket.  GES_OK once out_img is written
   (latency_ms, optional, receives submit-to-completion time), GES_ERR_NOT_READY when
   timeout_us == 0 and not done, GES_ERR_TIMEOUT when the wait ran out. */
ges_status ges_serve_poll(ges_server* srv, uint64_t ticket, int64_t timeout_us, float* latency_ms);

ges_status ges_serve_destroy(ges_server* srv);

#ifdef __cplusplus
}
#endif
#endif /* GES_H */
