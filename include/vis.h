/*
 * vis.h -- C ABI of the B300 (sm_103a) 3D Gaussian Splatting rasterizer.
 *
 * The library renders N 3D Gaussians to an image: preprocess (EWA projection,
 * spherical-harmonics colour, 3-sigma extent and tile overlap), duplication of
 * one (tile, depth) key per touched tile, a stable LSD radix sort of those keys,
 * per-tile ranges, and front-to-back alpha compositing; plus the adjoint of all of
 * it and a batched many-asset, many-camera form. The math is the paper's
 * definition of 3DGS (section 3.2): Eq. 1 (x_i = Pi(mu_i), S_i = J_i Sigma_i J_i^T),
 * Eq. 2 (w_i(x) = alpha_i exp(-1/2 (x-x_i)^T S_i^-1 (x-x_i))) and Eq. 3 (front-to-back
 * compositing in depth order), with the per-frame preprocess / GPU sort / draw
 * structure of Algorithm 1.
 *
 * Conventions (all calls):
 *  - Every pointer argument named as device memory must be a CUDA device pointer
 *    on the current device, 16-byte aligned, C-contiguous. Host pointers are
 *    named as such.
 *  - The caller owns all memory: inputs, outputs and the workspace. No call
 *    allocates device memory. A scene handle borrows the caller's attribute
 *    arrays (zero copy); they must outlive the handle and may be rewritten
 *    between frames.
 *  - Work is enqueued on the given stream and returns without synchronising,
 *    except vis_check(), which synchronises the stream. The kernels of a render are
 *    launched as programmatic dependents of their predecessor on the stream (each
 *    waits for it at entry, so ordering is unchanged; launches overlap tails); set
 *    the environment variable VIS_PDL=0 before the first call for plain launches.
 *  - Every call returns a vis_status; no exception or abort crosses the ABI.
 *    On failure, vis_last_error() returns a thread-local message.
 *  - Errors found on the device (key capacity exceeded, a bounded spin wait that
 *    ran out) are recorded in the workspace and returned by vis_check().
 */
#ifndef VIS_H
#define VIS_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define VIS_API __attribute__((visibility("default")))
#else
#define VIS_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    VIS_OK = 0,
    VIS_ERR_INVALID_ARG = 1,   /* rejected on the host; nothing was enqueued */
    VIS_ERR_CUDA = 2,          /* a CUDA runtime call failed */
    VIS_ERR_CAPACITY = 3,      /* more (tile, Gaussian) keys than the workspace holds */
    VIS_ERR_TIMEOUT = 4,       /* a bounded device spin wait gave up; outputs are invalid */
    VIS_ERR_UNSUPPORTED = 5
} vis_status;

/* Opaque scene handle: borrowed attribute pointers plus the SH degree. */
typedef struct vis_scene* vis_scene_t;

/* Pinhole camera, OpenCV axes (x right, y down, z forward).
 * A world point X maps to camera space as p = R X + t (R row-major), and to pixel
 * coordinates (fx p.x/p.z + cx, fy p.y/p.z + cy). Pixel (x, y) covers
 * [x, x+1) x [y, y+1); its centre is (x + 0.5, y + 0.5). Gaussians with
 * p.z <= near_z are culled (Algorithm 1, frustum cull). */
typedef struct {
    float R[9];
    float t[3];
    float fx, fy, cx, cy;
    float near_z;
} vis_camera;

/* Render options. Pass NULL for the defaults, or fill with vis_default_opts().
 *  tile        tile edge in pixels: 8, 16 or 32 (default 16)
 *  digit_bits  radix digit width of the depth-first order's 32-bit sorts (the depth sort
 *              of the surviving splats, and the tile sort of grids beyond the 16-bit path or
 *              of a batch): 8 (default), 10 or 11 bits per pass, i.e. 4, 4 or 3 passes over
 *              a depth. Wider digits mean fewer passes, each publishing 2^digit_bits
 *              look-back words per partition. sort_mode 0 and the 16-bit tile sort always
 *              use 8-bit digits. The order, hence the image, does not depend on it.
 *  dilation    low-pass term added to the diagonal of S (px^2, default 0.3)
 *  alpha_min   splats with alpha < alpha_min are skipped; Gaussians whose opacity
 *              is below it are culled (default 1/255)
 *  alpha_max   alpha is clamped to alpha_max (default 0.99)
 *  t_stop      compositing stops before the first splat that would bring the
 *              transmittance below t_stop (default 1e-4)
 *  sort_mode   how the (tile, depth, index) order is produced (Algorithm 1, "Radix Sort"):
 *              0 = one LSD sort of 64-bit (tile << 32 | depth) keys;
 *              1 = depth first (default): the surviving splats are sorted once by
 *                  32-bit depth (as in the paper), their tile copies are emitted in that
 *                  order and stably sorted by tile id alone. On grids of at most 51200
 *                  tiles the per-tile counts (hence ranges and digit histograms) come
 *                  first, the tile keys are 16-bit and the last pass writes only the
 *                  Gaussian indices;
 *              Both give the same order bit for bit; 1 moves about a quarter of the bytes
 *              of 0.
 *  pixels_per_thread  compositor block shape: 1 or 2 vertically adjacent pixels per
 *              thread (default 1); 2 evaluates both pixels with packed two-float
 *              arithmetic, rounded as the one-pixel code is: the image (and the adjoint's
 *              inputs) do not depend on it.
 *  collect_stats  1: the compositor also counts the (pixel, splat) pairs it tests and
 *              composites into vis_ctrl.pair_tests / hits (a few % slower); default 0.
 *  tile_extent which tiles a splat is listed in: 0 = every tile of the square of
 *              radius ceil(3 sqrt(lambda_max(S))) + 1 px around its centre; 1 = every
 *              tile of the tight box around the region where a pixel can take the splat
 *              (q <= min(9, 2 ln(opacity / alpha_min))); 2 (default) = that box with its
 *              top and bottom rows narrowed to the tiles whose band of pixel centres meets
 *              that region. The image does not depend on it; 1 lists ~40% fewer (tile,
 *              splat) pairs than 0, and 2 ~12% fewer than 1.
 *  spin_limit  how many times a sort partition (or a chunk of a block-sum scan, or a group
 *              of a partition's look-back) may poll a predecessor's unpublished
 *              look-back word before it gives up (0 = the default, 4194304; at most
 *              2^30). A wait that runs out records VIS_ERR_TIMEOUT in the workspace
 *              (returned by vis_check), publishes its own counts so that no other
 *              partition waits on it, and the render's later kernels skip their work and
 *              write NaN images; the workspace stays usable for the next render. The
 *              default only bounds a wait that can never end; small values exist to
 *              exercise that error path.
 * A splat reaches a pixel only inside its 3-sigma ellipse (Mahalanobis q <= 9). */
typedef struct {
    int tile;
    int digit_bits;
    float dilation;
    float alpha_min;
    float alpha_max;
    float t_stop;
    int sort_mode;
    int pixels_per_thread;
    int tile_extent;
    int collect_stats;
    int spin_limit;
} vis_render_opts;

VIS_API void vis_default_opts(vis_render_opts* opts);

/* Workspace layout (byte offsets from the workspace base), as used by
 * vis_render / vis_render_backward for a given (n, W, H, opts, ws_bytes).
 * Exposed so that callers can inspect intermediate stages. */
typedef struct {
    size_t total_bytes;      /* bytes the layout needs (<= ws_bytes) */
    int64_t key_capacity;    /* max (tile, Gaussian) keys the workspace holds */
    int tiles_x, tiles_y;
    int sort_passes;         /* radix passes over the key bits in use */
    int sorted_buffer;       /* 0 or 1: which key/val buffer holds the sorted result */
    size_t off_ctrl;         /* vis_ctrl, device-written status */
    size_t off_rec;          /* float4[n][3] splat records: (u,v,u_lo,v_lo), (f1,f2), (opacity,rgb) */
    size_t off_depth;        /* float[n] view depth (the sort key's low word) */
    size_t off_rect;         /* uint4[n] tile footprint: x0 | x1<<16, y0 | y1<<16 (the tile box,
                                upper bounds exclusive), row trims Lt | Rt<<8 | Lb<<16 | Rb<<24
                                (tiles dropped at the left / right ends of the top and bottom
                                rows, see tile_extent 2), 0 (a fused batch: the image) */
    size_t off_touched;      /* uint32[n] tiles touched (0 if culled) */
    size_t off_keys[2];      /* key_bytes x cap: sort keys (see key_bytes); with key_bytes 2 the
                                sorted keys are not stored (the tile of sorted position j is
                                the tile whose range holds j) */
    size_t off_vals[2];      /* uint32[cap] Gaussian index */
    size_t off_ranges;       /* uint2[tiles] [start, end) into the sorted keys */
    size_t off_tfinal;       /* float[H*W] final transmittance */
    size_t off_last;         /* int32[H*W] 1 + position, in the sorted key list, of the last composited splat (0 if none) */
    size_t off_g2;           /* float[n][9] screen-space gradients (backward scratch) */
    int key_bytes;           /* 8: (tile << 32) | depth bits (sort_mode 0); 4: tile id (sort_mode 1
                                beyond 51200 tiles); 2: 16-bit tile id (sort_mode 1) */
    int sort_mode;
    size_t off_order;        /* key_bytes 2 only (else 0): uint32[tiles], the order in which the
                                compositor and its adjoint take the tiles -- a permutation of the
                                tiles by non-increasing key count, in log-spaced buckets of two
                                per octave (ties in any order); the image does not depend on it */
} vis_ws_layout;

/* Device-written status block at workspace offset off_ctrl (= 0). */
typedef struct {
    uint32_t num_keys;       /* (tile, splat) pairs listed by the last render (may exceed capacity) */
    uint32_t error;          /* bit 0: capacity exceeded, bit 1: spin timeout, bit 2: an adjoint asked
                                of a dynamic frame (vis_render_dynamic) */
    uint32_t internal[16];   /* sort partition tickets */
    uint32_t num_visible;    /* Gaussians that survived culling (sort_mode 1) */
    uint32_t flags;          /* bit 0: the last render was a dynamic frame (it has no adjoint) */
    uint64_t pair_tests;     /* with collect_stats: (pixel, splat) pairs the compositor tested */
    uint64_t hits;           /* with collect_stats: pairs it composited */
    uint32_t internal2[2];   /* block-sum scan tickets */
    uint32_t reserved[38];
} vis_ctrl;

/* Borrow a scene (section 3.2: mean, scale, rotation quaternion, opacity, SH colour).
 *  means          device float[n][3]
 *  log_scales     device float[n][3]   s = exp(log_s)
 *  quats          device float[n][4]   (w, x, y, z); normalised by the renderer
 *  opacity_logits device float[n]      opacity = sigmoid(logit)
 *  sh             device float[n][K][3], K = (sh_degree+1)^2, coefficient k = l*l+l+m
 *  sh_degree      0..3
 *  n              1 .. 2^31-1
 * Errors: VIS_ERR_INVALID_ARG for null/misaligned pointers or bad sizes. */
VIS_API vis_status vis_scene_upload(const float* means, const float* log_scales, const float* quats,
                            const float* opacity_logits, const float* sh, int sh_degree,
                            int64_t n, vis_scene_t* out);
VIS_API void vis_scene_destroy(vis_scene_t scene);

/* Pre-packed FP16 scenes (Algorithm 1, "Pre-pack (only once)"; section 3.4, "Pre-pack and
 * FP16 layout": the covariance is formed once from scale and rotation, and mean, opacity,
 * the covariance's upper triangle and the colour are cast to fp16 and packed two per
 * 32-bit word to halve the per-frame attribute bytes). Three device planes per scene,
 * every value an IEEE half, two per uint32 word, the first in the low 16 bits:
 *  pos  uint32[n][2]  (mu_x, mu_y), (mu_z, alpha)      alpha = sigmoid(logit), the opacity
 *  cov  uint32[n][3]  (xx, xy), (xz, yy), (yz, zz)     Sigma = R diag(s)^2 R^T, upper triangle
 *  col  uint32[n][W]  the SH coefficients in the order of vis_scene_upload's sh array,
 *                     zero-padded; W = 3 (sh_degree+1)^2 halves rounded up to an even
 *                     number of words (W = 2, 6, 14, 24 for degrees 0..3)
 * vis_packed_size gives each plane's bytes (any pointer may be NULL). vis_scene_pack fills
 * the planes from an fp32 scene on `stream` (covariance and sigmoid in float, then rounding
 * to nearest even). vis_scene_upload_packed borrows planes (16-byte aligned) as a scene that
 * every render call accepts (vis_render, vis_render_depth, vis_render_multi, the batch);
 * its preprocess reads about half the bytes. Values must lie in the fp16 range; a packed
 * scene has no parameter gradients (the backward calls return VIS_ERR_UNSUPPORTED).
 * Errors: VIS_ERR_INVALID_ARG for null/misaligned pointers, bad sizes, or packing a packed
 * scene. */
VIS_API vis_status vis_packed_size(int64_t n, int sh_degree, size_t* pos_bytes, size_t* cov_bytes,
                                   size_t* col_bytes);
VIS_API vis_status vis_scene_pack(vis_scene_t scene, void* pos, void* cov, void* col, void* stream);
VIS_API vis_status vis_scene_upload_packed(const void* pos, const void* cov, const void* col,
                                           int sh_degree, int64_t n, vis_scene_t* out);

/* Bytes of workspace vis_render needs for n Gaussians at W x H holding up to
 * key_capacity (tile, Gaussian) keys (one per tile a splat's rectangle touches). */
VIS_API vis_status vis_workspace_size(int64_t n, int W, int H, int64_t key_capacity,
                              const vis_render_opts* opts, size_t* bytes);

/* Layout of a workspace of ws_bytes for (n, W, H, opts); key_capacity is the
 * largest that fits. VIS_ERR_INVALID_ARG if ws_bytes cannot hold even one key. */
VIS_API vis_status vis_workspace_layout(int64_t n, int W, int H, size_t ws_bytes,
                                const vis_render_opts* opts, vis_ws_layout* out);

/* Forward render of one view (section 3.2 Eqs. 1-3; Algorithm 1 per-frame path).
 *  bg         host float[3] background colour
 *  out_rgb    device float[3][H][W] (planar)
 *  out_alpha  device float[H][W] = 1 - final transmittance
 *  ws         device workspace of ws_bytes (>= vis_workspace_size for the keys produced);
 *             it keeps the intermediates that vis_render_backward reads
 *  stream     cudaStream_t (NULL = legacy default stream)
 * Device-side errors are reported by vis_check(). */
VIS_API vis_status vis_render(vis_scene_t scene, const vis_camera* cam, int W, int H, const float bg[3],
                      float* out_rgb, float* out_alpha, void* ws, size_t ws_bytes,
                      const vis_render_opts* opts, void* stream);

/* Synchronise `stream`, read the status block of `ws`, and return VIS_OK,
 * VIS_ERR_CAPACITY or VIS_ERR_TIMEOUT. num_keys (host, may be NULL) receives the
 * number of keys the last render produced (the capacity a retry needs). */
VIS_API vis_status vis_check(const void* ws, void* stream, int64_t* num_keys);

/* Adjoint of vis_render (section 3.2: the splatting formulation is differentiable
 * in all Gaussian parameters). Must follow a vis_render with the same scene
 * contents, camera, size, bg, opts and workspace.
 *  d_rgb, d_alpha   device float[3][H][W], float[H][W]: dL/d out_rgb, dL/d out_alpha
 *  d_means .. d_sh  device outputs shaped like the scene arrays; overwritten
 * Decision sets (culling, the 3-sigma cut, the alpha_min skip, the early stop)
 * are held fixed; the alpha_max clamp and the colour clamp at 0 pass no gradient. */
VIS_API vis_status vis_render_backward(vis_scene_t scene, const vis_camera* cam, int W, int H,
                               const float bg[3], const float* d_rgb, const float* d_alpha,
                               void* ws, size_t ws_bytes, const vis_render_opts* opts,
                               float* d_means, float* d_log_scales, float* d_quats,
                               float* d_opacity_logits, float* d_sh, void* stream);

/* Depth-buffer-aware compositing (section 3.4: the splats are drawn against the depth of
 * opaque geometry with the depth test on and depth writes off). As vis_render, plus
 *  depth   device float32 [H,W] (row-major, 16-byte aligned, not modified): per pixel,
 *          a view depth (camera-space z, the units of the splat depths); a splat whose
 *          view depth exceeds it is not composited at that pixel (+inf and NaN test
 *          nothing, so an all-inf buffer gives vis_render's image bit for bit; -inf
 *          rejects every splat).
 * The buffer also culls work without changing any pixel: a small kernel takes each tile's
 * largest value, the preprocess drops a splat deeper than that in every tile it reaches
 * (so it is neither sorted nor listed), and the compositor skips splats deeper than all
 * of a pixel block's values.
 * Errors: as vis_render, and VIS_ERR_INVALID_ARG for a null or misaligned depth. */
VIS_API vis_status vis_render_depth(vis_scene_t scene, const vis_camera* cam, int W, int H,
                                    const float bg[3], const float* depth, float* out_rgb,
                                    float* out_alpha, void* ws, size_t ws_bytes,
                                    const vis_render_opts* opts, void* stream);

/* The adjoint of vis_render_depth (the same depth buffer, after vis_render_depth on the same
 * workspace): as vis_render_backward, with the depth test among the held decisions. */
VIS_API vis_status vis_render_backward_depth(vis_scene_t scene, const vis_camera* cam, int W, int H,
                                             const float bg[3], const float* depth, const float* d_rgb,
                                             const float* d_alpha, void* ws, size_t ws_bytes,
                                             const vis_render_opts* opts, float* d_means,
                                             float* d_log_scales, float* d_quats,
                                             float* d_opacity_logits, float* d_sh, void* stream);

/* Several scenes ("models") composited into one image (Algorithm 1: every model is
 * preprocessed under its own affine transform M_k, then ONE radix sort and one compositing
 * pass run over the splats of all models, so that splats of different models interleave
 * in depth -- the order a per-model sort cannot give; section 3.4).
 *  scenes    host array of n_scenes scene handles (1..65536); the same handle may appear
 *            more than once (instancing)
 *  models    host float [n_scenes][12], or NULL for identity transforms: row-major 3x4
 *            [A | b]; model k draws its Gaussians at A mu + b with covariance A Sigma A^T,
 *            and evaluates their SH colour along the view ray mapped back into the
 *            model's own frame (A^-1 (x - camera centre)), so that a rigidly moved model
 *            keeps its view-dependent appearance. A must be invertible.
 *  depth     device float32 [H,W] depth buffer as in vis_render_depth, or NULL
 *  ws        a workspace sized for n = vis_multi_slots(scenes, n_scenes): scene k occupies
 *            the slots [offset_k, offset_k + n_k), offset_k = sum over j < k of n_j rounded
 *            up to 256 (the slot of model k's Gaussian i is offset_k + i; the padding
 *            slots are never listed)
 * Otherwise as vis_render / vis_render_depth. Errors: VIS_ERR_INVALID_ARG for a null
 * scene, a non-finite or singular model, or more than 2^31-1 slots. */
VIS_API vis_status vis_multi_slots(const vis_scene_t* scenes, int n_scenes, int64_t* slots);
VIS_API vis_status vis_render_multi(const vis_scene_t* scenes, const float* models, int n_scenes,
                                    const vis_camera* cam, int W, int H, const float bg[3],
                                    const float* depth, float* out_rgb, float* out_alpha, void* ws,
                                    size_t ws_bytes, const vis_render_opts* opts, void* stream);

/* Gradient outputs of one scene (device, shaped like the scene's arrays, overwritten). */
typedef struct {
    float* d_means;
    float* d_log_scales;
    float* d_quats;
    float* d_opacity_logits;
    float* d_sh;
} vis_scene_grads;

/* The adjoint of vis_render_multi (same scenes, models, camera, depth, opts and workspace,
 * after vis_render_multi): gradients with respect to each model's own, untransformed
 * parameters. grads: host array of n_scenes gradient sets; a scene handle listed twice
 * needs two distinct gradient sets (their sum is the handle's gradient). */
VIS_API vis_status vis_render_backward_multi(const vis_scene_t* scenes, const float* models,
                                             int n_scenes, const vis_camera* cam, int W, int H,
                                             const float bg[3], const float* depth,
                                             const float* d_rgb, const float* d_alpha, void* ws,
                                             size_t ws_bytes, const vis_render_opts* opts,
                                             const vis_scene_grads* grads, void* stream);

/* Stable LSD radix sort of (key, value) pairs on the device: the sort stage of the
 * renderer (Algorithm 1, "Radix Sort"; section 3.4, GPU sorting) exposed on its own.
 *  keys_in, vals_in    device uint64[m], uint32[m] (not modified)
 *  keys_out, vals_out  device uint64[m], uint32[m]
 *  key_bits            only bits [0, key_bits) take part (1..64); higher bits must be 0
 *  ws                  device workspace of vis_sort_workspace_size(m, key_bits) bytes
 * Equal keys keep their input order. */
VIS_API vis_status vis_sort_workspace_size(int64_t m, int key_bits, size_t* bytes);
VIS_API vis_status vis_sort_pairs(const uint64_t* keys_in, const uint32_t* vals_in, uint64_t* keys_out,
                          uint32_t* vals_out, int64_t m, int key_bits, void* ws, size_t ws_bytes,
                          void* stream);

/* Batched render of many assets seen by many cameras (the paper renders several models
 * per frame with one global radix sort, Algorithm 1 "for all model M_k", section 3.4);
 * every (asset, camera) pair is an independent image. A batch handle is created with
 * `lanes`:
 *  lanes = 0   one fused pipeline: one preprocess launch over the work list of items (each
 *              image's Gaussians in their own run of workspace slots); the images are
 *              grouped, the widest first, and a group's images stacked as tile rows of one
 *              canvas (a tile grid as wide as its widest image, at most 51200 tiles); each
 *              group then runs the single-image pipeline over its canvas -- one depth sort of
 *              the survivors of all its images, the tile copies emitted in that order with
 *              canvas tile ids, the counts-first stable sort by that id (i.e. by image and
 *              tile, keeping depth order inside each tile) and one compositor launch over the
 *              canvas. It always uses the depth-first order (opts->sort_mode is ignored);
 *              opts->tile, digit_bits and pixels_per_thread apply to every image. The groups
 *              run on three streams, each with a scratch area: key_capacity bounds the tile
 *              copies of each group (the copies of all images together always suffice). Each image is bit-identical to
 *              vis_render of the same (asset, camera, options).
 *  lanes >= 1  per-image vis_render calls on that many streams forked from the batch's
 *              origin stream (longest-processing-time assignment of images to lanes), each
 *              lane in its own workspace slice of key_capacity keys.
 * In both forms the whole launch sequence is captured into a CUDA graph on the first call
 * and replayed by later calls with identical arguments (same pointers, cameras, sizes,
 * options); the fused form also copies its item tables (a few hundred bytes per image)
 * from host memory into the workspace before every launch.
 *  scenes[n_scenes]        scene handles (host array; plain or pre-packed)
 *  cams[n_images]          host array of cameras; cam_scene[i] = asset of image i
 *  W, H[n_images]          host arrays of image sizes
 *  out_rgb, out_alpha      host arrays of n_images device pointers ([3][H][W], [H][W])
 *  ws, ws_bytes            device workspace >= vis_batch_workspace_size(...) (256-byte
 *                          aligned for lanes = 0); at most 65536 images and 2^31-1
 *                          Gaussian slots in a fused batch
 * The first call synchronises nothing but must not itself be inside a stream capture.
 * Device errors of any image are returned by vis_batch_check (which synchronises); its
 * max_keys is the largest image's key count (lanes >= 1) or the largest group's (lanes = 0),
 * the capacity a retry needs. */
typedef struct vis_batch* vis_batch_t;
VIS_API vis_status vis_batch_create(int lanes, vis_batch_t* out);
VIS_API void vis_batch_destroy(vis_batch_t batch);
VIS_API vis_status vis_batch_workspace_size(const vis_scene_t* scenes, int n_scenes, const int* cam_scene,
                                            const int* W, const int* H, int n_images, int lanes,
                                            int64_t key_capacity, const vis_render_opts* opts,
                                            size_t* bytes);
VIS_API vis_status vis_render_batch(vis_batch_t batch, const vis_scene_t* scenes, int n_scenes,
                                    const vis_camera* cams, const int* cam_scene, const int* W,
                                    const int* H, int n_images, const float bg[3],
                                    float* const* out_rgb, float* const* out_alpha, void* ws,
                                    size_t ws_bytes, const vis_render_opts* opts, void* stream);
VIS_API vis_status vis_batch_check(const void* ws, int n_images, void* stream, int64_t* max_keys);

/* Per-frame update of a dynamic scene (stands in for the per-frame Gaussian
 * generator of section 3.3; the renderer re-sorts globally every frame, section 4):
 *   means_out[i]  = means0[i] + t velocity[i]
 *   logits_out[i] = logits0[i] + amp[i] sin(2 pi freq[i] t + phase[i])
 *  means0, velocity      device float[n][3]
 *  logits0, amp, freq, phase  device float[n]
 *  means_out, logits_out device float[n][3], float[n] (may be the arrays a scene borrows)
 * Outputs must not alias the inputs. */
VIS_API vis_status vis_dynamic_update(const float* means0, const float* velocity, const float* logits0,
                                      const float* amp, const float* freq, const float* phase, float t,
                                      int64_t n, float* means_out, float* logits_out, void* stream);

/* Frame t of a dynamic scene without storing it: `scene` borrows the frame-0 attributes
 * (its means and opacity_logits are means0 and logits0 above), and the preprocess applies
 * vis_dynamic_update's formulas to them as it reads them, rounding exactly as that kernel
 * does; the image is the one vis_dynamic_update into a scene followed by vis_render of it
 * gives, bit for bit, without the update's 16 B per Gaussian written and read back.
 *  velocity            device float[n][3]   (n = the scene's size)
 *  amp, freq, phase    device float[n]
 * Plain fp32 scenes only (VIS_ERR_UNSUPPORTED for a pre-packed scene). The frame has no
 * adjoint: a vis_render_backward on its workspace computes nothing, and vis_check then
 * returns VIS_ERR_UNSUPPORTED (status bit 2) until the next render. Other arguments and
 * errors as vis_render. */
VIS_API vis_status vis_render_dynamic(vis_scene_t scene, const float* velocity, const float* amp,
                                      const float* freq, const float* phase, float t, const vis_camera* cam,
                                      int W, int H, const float bg[3], float* out_rgb, float* out_alpha,
                                      void* ws, size_t ws_bytes, const vis_render_opts* opts, void* stream);

/* The same sort for callers that cannot allocate device memory (the paper has no
 * counterpart; this is a library convenience). Some callers may not call cudaMalloc
 * where they sort -- a real-time loop with a fixed memory budget, a plug-in whose
 * host application owns all device allocations, code that must not risk the device
 * synchronisation an allocation can cause -- so they cannot pass the workspace
 * vis_sort_pairs needs. This entry point allocates nothing: its scratch is a fixed
 * array of VIS_SORT_NOALLOC_SCRATCH_BYTES (about 16 MiB) of static device memory
 * inside the library, which every GPU that loads the library holds until the
 * process exits. The caller still passes the inputs and outputs, as for
 * vis_sort_pairs (same layout, alignment and stability).
 *  m          0 .. VIS_SORT_NOALLOC_MAX_KEYS; larger m returns VIS_ERR_INVALID_ARG
 *  key_bits   1..64
 * The first call on a device, with that device current, looks up the array's
 * device address (cudaGetSymbolAddress) and caches it; make that first call before
 * any stream capture; a device reset (cudaDeviceReset) after that first call is not
 * supported, since the cached address may no longer be the array's. Every call shares
 * the one array (it is cleared where needed at the start of each call), so calls whose
 * GPU work overlaps -- on different streams, or from different threads -- race and
 * must be serialised by the caller.
 * A device-side error of the sort (a look-back wait that ran out, VIS_ERR_TIMEOUT: the
 * outputs are then invalid) is kept in the array's status word until the next call;
 * vis_sort_noalloc_check(stream) synchronises `stream` and returns it (it allocates
 * nothing either). The same error of vis_sort_pairs is read with vis_check(ws, ...),
 * its workspace starting with the same status block. */
#define VIS_SORT_NOALLOC_MAX_KEYS (1 << 20)
#define VIS_SORT_NOALLOC_SCRATCH_BYTES 17047808
VIS_API vis_status vis_sort_pairs_noalloc(const uint64_t* keys_in, const uint32_t* vals_in,
                                          uint64_t* keys_out, uint32_t* vals_out, int64_t m,
                                          int key_bits, void* stream);
VIS_API vis_status vis_sort_noalloc_check(void* stream);

/* Per-stage timing of vis_render (tracing; the paper times its frame by stages,
 * Table 1 "Sort" vs "Prep.+Draw"). Between vis_profile_begin and vis_profile_end,
 * every vis_render records CUDA events on its stream between its stages, for up
 * to 1024 renders. vis_profile_end synchronises those events and returns, per
 * stage, the summed milliseconds over the recorded renders, in this order:
 *   0 clear, 1 preprocess,
 *   sort_mode 1: 2 compaction + depth sort, 3 emission of the tile copies in depth order,
 *                4 per-tile counts (or the tile histogram), 5 tile digit passes;
 *   sort_mode 0: 2 scan + key duplication, 3 sort histogram, 4 (empty), 5 digit passes;
 *   6 tile ranges (empty when the counts produced them), 7 composite.
 *  stage_ms   host double[max_stages]
 *  n_stages   host out: number of stages written (8)
 *  n_renders  host out: renders summed
 *  n_passes   host out: radix passes per render (of the last render)
 * Profiling is per process and not thread safe. */
VIS_API vis_status vis_profile_begin(void);
VIS_API vis_status vis_profile_end(double* stage_ms, int max_stages, int* n_stages, int* n_renders,
                                   int* n_passes);

/* Thread-local description of the last error (empty string if none). */
VIS_API const char* vis_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* VIS_H */
