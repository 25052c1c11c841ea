/*
 * splotch.h: C ABI of the GB300 (sm_103a) Splotch hot path.
 *
 * Method: Dykes, Gheller, Rivi, Krokos, "Splotch: porting and optimizing for the
 * Xeon Phi".  A frame is: per-particle rasterisation (roto-translation and perspective
 * projection with reference to a camera and look-at point, clipping, colour from a
 * scalar through a runtime colormap; Section 2.1, Section 3.1), binning of particles
 * into square image tiles with the rule "distance to tile centre < 0.75 radius +
 * sqrt(2) tile / 2" (Section 3.2.1, tile-list pseudocode), and per-tile accumulation
 * of each particle's Gaussian footprint, colour times scalar weight (Section 2.1,
 * Section 3.2.2), followed by the per-pixel final transform.  The mode built here is
 * absorption equal to emission, whose radiative-transfer update (Section 2.1) closes
 * to O = 1 - exp(-a) with a the additive accumulation.
 *
 * Conventions fixed by this library where the paper is silent:
 *   camera: right-handed, vertical field of view, up vector projected out of the view
 *     direction; pixel (i, j) has its centre at (i + 0.5, j + 0.5), row 0 at the top;
 *   screen radius r = F h / z_c, support R = max(rfac r, r_min_px), Gaussian
 *     sigma = sigma_over_R R truncated at distance < R (defaults 0.75, 0.75 px, 0.5);
 *   colormap: linear interpolation between entries, emission = brightness x colour;
 *   images: float32, row-major H x W x 3 (RGB interleaved).
 *   Every decision that turns floating point into an integer (near-plane cull, pixel
 *   coverage, tile membership) is evaluated in FP32 with each operation rounded once
 *   to nearest-even and no fused multiply-add, in the order written in the comments
 *   of splotch_render below; values (colours, weights, sums) are FP32.
 *
 * Errors: every call returns a status; nothing throws across the ABI.  On failure
 * splotch_last_error() gives a one-line reason for the calling thread.
 * Threading: a scene is read-only after creation and may be rendered concurrently
 * from several host threads on different streams; each render call allocates its own
 * workspace.  Calls on one plan must not overlap.
 */
#ifndef SPLOTCH_H
#define SPLOTCH_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct splotch_scene splotch_scene; /* opaque, library-owned device-resident particles */
typedef struct splotch_plan splotch_plan;   /* opaque, pre-sized multi-view render */

typedef enum {
    SPLOTCH_OK = 0,
    SPLOTCH_ERR_INVALID_ARG = 1, /* rejected before any GPU work */
    SPLOTCH_ERR_OOM = 2,         /* an allocation (callback or default) returned NULL */
    SPLOTCH_ERR_CUDA = 3,        /* a CUDA runtime call failed */
    SPLOTCH_ERR_CAPACITY = 4,    /* a plan's pre-sized buffers were too small for this frame */
    SPLOTCH_ERR_TIMEOUT = 5,     /* a bounded device wait ran out (the kernel returned early) */
    SPLOTCH_ERR_UNSUPPORTED = 6  /* valid request outside this build's limits (e.g. tile count) */
} splotch_status;

typedef enum { SPLOTCH_F32 = 0, SPLOTCH_F16 = 1, SPLOTCH_BF16 = 2 } splotch_storage;

/* Device memory provider for scene storage and per-call workspaces.  alloc returns a
 * device pointer aligned to at least 256 bytes (or NULL: the call fails with
 * SPLOTCH_ERR_OOM); both callbacks are stream-ordered on `stream` (a cudaStream_t).
 * All-NULL fields select the library's own stream-ordered memory pool. */
typedef struct {
    void *(*alloc)(void *ctx, size_t bytes, void *stream);
    void (*free)(void *ctx, void *ptr, void *stream);
    void *ctx;
} splotch_allocator;

/* Particle set (Section 2.1: positions, an intrinsic radius per particle, a scalar
 * field mapped through a runtime colormap; Section 4.1: gas and star species).
 * Species are contiguous index ranges [type_begin[t], type_begin[t+1]).
 *   n            particle count, >= 0
 *   n_types      1..255
 *   type_begin   host, n_types + 1 entries, type_begin[0] = 0, non-decreasing, last = n
 *   x y z h intensity   n floats each (FP32), on the device when on_device != 0, else host;
 *                h > 0 (smoothing length, world units); all finite.  Host inputs that
 *                are all page-locked (cudaHostAlloc / cudaHostRegister) are read in place
 *                by the device; pageable host inputs are first copied to device staging
 *   storage      splotch_storage for the resident copy of x, y, z, h and the normalised
 *                intensity (FP16 / BF16 round to nearest even from FP32)
 *   cmap_rgb     host, per type a pointer to cmap_len[t] RGB triples (FP32), cmap_len >= 2
 *   brightness   host, per type (emission = brightness x colour)
 *   i_log        host, per type: 1 = take ln(max(I, 1e-30)) before ranging
 *   i_min i_max  host, per type range of the (logged) intensity; NULL = the exact min / max
 *                over the species (Section 2.1: ranging and normalisation).  The normalised
 *                intensity clamp((I' - i_min) / (i_max - i_min), 0, 1), or 0 when
 *                i_max <= i_min, selects the colour.
 *   allocator    see splotch_allocator; stream: cudaStream_t used for the copies.
 * Inputs may be freed once splotch_create_scene returns (it synchronises `stream`). */
typedef struct {
    int64_t n;
    int32_t n_types;
    const int64_t *type_begin;
    const float *x, *y, *z, *h, *intensity;
    int32_t on_device;
    int32_t storage;
    const float *const *cmap_rgb;
    const int32_t *cmap_len;
    const float *brightness;
    const float *i_min;
    const float *i_max;
    const int32_t *i_log;
    splotch_allocator allocator;
    void *stream;
    /* Colour from a vector field (Section 2.1: colours come directly from a vector input
     * field, or from a scalar through a colormap).  col_vector: NULL (every species uses
     * its colormap), or host, per type: nonzero = the species' colour is the particle's RGB
     * triple.  rgb: n x 3 floats (r, g, b interleaved), where on_device says (host input
     * may be pageable or page-locked); read for the particles of vector-coloured species,
     * which must be finite, and ignored elsewhere.  A vector species' components are
     * ranged and normalised like the intensity, with its i_log and one range over its
     * three components (i_min / i_max, or their joint min / max): emission = brightness x
     * (r~, g~, b~); its intensity is not used.  The scene then holds a per-particle FP32
     * emission (16 bytes per particle, whatever the storage) and its tile records carry
     * particle indices. */
    const int32_t *col_vector;
    const float *rgb;
} splotch_scene_desc;

/* Camera (Section 2.1: supplied camera and look-at positions, then clipping).  FP64 on
 * the host; the library composes f = (L - E)/|L - E|, s = (f x U)/|f x U|, u = s x f,
 * rows (s, u, f) with translations -(row . E), and F = (0.5 H) / tan(fov_deg pi / 360),
 * then rounds each to FP32 (the only FP64 step).  A particle is visible for
 * z_near < zc <= z_far (FP32 zc and planes); z_far 0 or not finite: no far plane.
 * Cameras that differ only in (z_near, z_far) = consecutive bounds cut the particles
 * into depth slabs, each particle in exactly one.  Rejected: width or height < 1, fov
 * outside (0, 180), z_near <= 0, a far plane at or before z_near, eye == lookat,
 * |f x U| <= 1e-9 |U|. */
typedef struct {
    double eye[3], lookat[3], up[3];
    double fov_deg; /* vertical field of view, degrees */
    double z_near;  /* particles with camera depth <= z_near are culled */
    int32_t width, height;
    double z_far;   /* particles with camera depth > z_far are culled; 0: no far plane */
} splotch_camera;

/* Render parameters.
 *   tile          square tile edge in pixels, 1..64, with at most 16384 tiles per image;
 *                 0 = 16 (or the smallest edge above 16, in steps of 8, that meets
 *                 the tile limit).
 *                 Section 3.1: the tile size is a runtime parameter.
 *   rfac          support radius factor, > 0 (0.75; Section 3.2.1 threshold)
 *   sigma_over_R  Gaussian sigma as a fraction of the support, > 0 (0.5)
 *   r_min_px      smallest support radius in pixels, >= 0 (0.75)
 *   block_particles  particles each CTA of the raster / count / scatter kernels streams,
 *                 rounded up to a multiple of 1024 (FP32) or 2048 (FP16 / BF16);
 *                 0 = about four CTAs per SM.  A tuning knob with no effect on results.
 *   flags         SPLOTCH_OUT_ACCUM: write the accumulation a instead of 1 - exp(-a);
 *                 SPLOTCH_OUT_ADD: add the accumulation a to what `out` holds (several
 *                 renders, e.g. particle subsets, summed in one image; the final transform
 *                 is then applied once with splotch_final_transform);
 *                 SPLOTCH_SYNC: splotch_render waits for the frame and reports a device-side
 *                 TIMEOUT before returning; SPLOTCH_PLAN_GRAPH: a plan captures its launch
 *                 sequence into a CUDA graph on first launch and replays it afterwards;
 *                 SPLOTCH_TIMING: splotch_render records CUDA events around each kernel on
 *                 `stream`, waits for the frame and keeps the durations for
 *                 splotch_last_timing; SPLOTCH_STABLE: build every tile list in ascending
 *                 particle index (Section 3.2.1 fills each thread's index vectors by walking
 *                 its particles in order), which makes the image bitwise reproducible; the
 *                 binning takes about three times as long.  Without it a list holds the
 *                 same members, each chunk's in the order its warps reached them, and two
 *                 renders may differ by the FP32 rounding of a pixel's sum in another order
 *                 (at most 2 (n - 1) 2^-24 of the sum, n its contributions). */
typedef struct {
    int32_t tile;
    float rfac;
    float sigma_over_R;
    float r_min_px;
    int32_t block_particles;
    int32_t flags;
} splotch_render_params;

enum {
    SPLOTCH_OUT_ACCUM = 1, SPLOTCH_SYNC = 2, SPLOTCH_PLAN_GRAPH = 4, SPLOTCH_TIMING = 8, SPLOTCH_OUT_ADD = 16,
    SPLOTCH_OUT_MAP = 32, /* splotch_render_ordered: write the per-pixel affine map (alpha, beta) */
    SPLOTCH_STABLE = 64   /* tile lists in ascending particle index: bitwise reproducible images */
};

/* Defaults listed above. */
splotch_render_params splotch_default_params(void);

/* Copy a particle set to the device (library-owned), normalise the intensity per species
 * (Section 2.1 preprocessing) and store the attributes in the requested precision.
 * Errors: INVALID_ARG (bad counts, ranges, pointers, colormaps, non-finite or h <= 0),
 * OOM, CUDA.  *out is set only on success. */
splotch_status splotch_create_scene(const splotch_scene_desc *desc, splotch_scene **out);

/* Release a scene (NULL is accepted).  The caller guarantees no render on it is in flight. */
splotch_status splotch_destroy(splotch_scene *scene);

/* Scene facts: particle count, species count, storage, device bytes held. */
splotch_status splotch_scene_info(const splotch_scene *scene, int64_t *n, int32_t *n_types,
                                  int32_t *storage, int64_t *device_bytes);

/* The FP32 camera parameters the kernels use: m = 3x4 row-major view matrix,
 * p = {F, W/2, H/2, z_near, z_far (+infinity without a far plane)}.  Host only. */
splotch_status splotch_camera_params(const splotch_camera *cam, float m[12], float p[5]);

/* Render n_views >= 1 frames of one scene into out (device, n_views x H x W x 3 FP32; all
 * cameras the same size).  Per view, per particle (FP32, each operation rounded once):
 *   xc = ((m0 x + m1 y) + m2 z) + m3 (rows 1, 2 likewise), visible iff z_near < zc <= z_far;
 *   X = W/2 + (F xc)/zc, Y = H/2 - (F yc)/zc, r = (F h)/zc, R = max(rfac r, r_min_px);
 *   pixel box i in [max(0, ceil(clamp((X - R) - 0.5, -2, W + 1)) - 1),
 *                   min(W - 1, floor(clamp((X + R) - 0.5, -2, W + 1)) + 1)], rows likewise;
 *   pixel (i, j) covered iff in the box and ((i + .5) - X)^2 + ((j + .5) - Y)^2 < R R;
 *   tile (tx, ty) of edge T holds the particle iff it meets the box and
 *     (cx - X)^2 + (cy - Y)^2 < (R + 0.70710677 T)^2, cx = (tx + .5) T, cy = (ty + .5) T;
 *   a(i, j) = sum over covered particles of e exp(-d^2 / (sigma_over_R R)^2);
 *   out = 1 - exp(-a) (or a with SPLOTCH_OUT_ACCUM).
 * The call blocks until the particle-tile pair count of each view is known (to size the
 * tile lists), then enqueues the rest on `stream` and returns; out is ready when `stream`
 * reaches that point.  Errors: INVALID_ARG, UNSUPPORTED, OOM, CUDA, TIMEOUT. */
splotch_status splotch_render(splotch_scene *scene, const splotch_camera *cams, int32_t n_views,
                              const splotch_render_params *params, float *out, void *stream);

/* Depth-ordered render of one view with absorption different from emission (Section 2.1:
 * the image solves the radiative-transfer equation along each line of sight).  Particles
 * of species t absorb A = absorb[t] x E (absorb: host, n_types floats, finite, >= 0) and
 * are applied from the farthest to the nearest (z_c descending) from a black background:
 * I <- I exp(-A w) + (E / A)(1 - exp(-A w)), or I <- I + E w where A = 0.  out: device,
 * H x W x 3 FP32, receives I (no final transform: with absorb[t] = 1 for every species I
 * equals 1 - exp(-a) of splotch_render).  With SPLOTCH_OUT_MAP in params->flags, out is
 * H x W x 6 and receives, per pixel, the affine map the particles apply to the intensity
 * entering from behind, I_out = alpha I_in + beta: (alpha_r, alpha_g, alpha_b, beta_r,
 * beta_g, beta_b), alpha the product of exp(-A w) and beta the I above; the maps of
 * depth slabs (cameras with consecutive near / far planes) compose far to near into the
 * whole frame.  Particles at exactly equal depth are applied in index order.  Tiles up
 * to 32 px (larger: UNSUPPORTED); other output flags are ignored.  The particles are sorted by
 * depth (stable radix sort from index order), their records written out in that order and
 * grouped by a stable sort on tile id; device memory besides the tile lists: about 52
 * bytes per particle and 32 per particle-tile pair.  Synchronous.  Errors: INVALID_ARG,
 * UNSUPPORTED, OOM, CUDA, TIMEOUT. */
splotch_status splotch_render_ordered(splotch_scene *scene, const splotch_camera *cam,
                                      const splotch_render_params *params, const float *absorb, float *out,
                                      void *stream);

/* Out-of-core render of one view (Section 3.1: data sets larger than the accelerator's memory
 * go through it in double-buffered pieces, transfers overlapping work).  The particle set `desc` stays where it is (host or device, as for
 * splotch_create_scene) and is rendered in chunks of at most `chunk` particles (the first
 * a sixth of `chunk`, at least 2^20 particles, each next one 3/2 of the last, so that the
 * first transfer is short): each chunk is prepared on the device on a side stream while
 * the previous chunk renders on `stream`, and its accumulation is added to `out`.  With
 * absorption = emission the accumulation is a sum over particles, so the result equals
 * splotch_render of the whole set up to FP32 summation order.  Intensity ranges not given
 * are computed exactly over the whole set first (one extra pass over the intensities).
 * Flags: SPLOTCH_OUT_ACCUM leaves the accumulation a in `out`; SPLOTCH_OUT_ADD adds it to
 * what `out` holds; otherwise `out` = 1 - exp(-a).  Device memory: two chunks' resident
 * attributes plus one chunk's frame workspace.  Synchronous: returns when `out` is ready.
 * Errors: as splotch_create_scene and splotch_render; INVALID_ARG if chunk < 1. */
splotch_status splotch_render_streamed(const splotch_scene_desc *desc, int64_t chunk, const splotch_camera *cam,
                                       const splotch_render_params *params, float *out, void *stream);

/* Final transform in place: a[k] <- 1 - exp(-a[k]) for k < count (device FP32 buffer).
 * With SPLOTCH_OUT_ACCUM renders this finishes an accumulation image, e.g. after the
 * accumulations of several particle shards have been summed (the mode is additive,
 * Section 2.1 and Section 3.2.2).  Asynchronous on `stream`; INVALID_ARG for count < 0. */
splotch_status splotch_final_transform(float *a, int64_t count, void *stream);

/* Composition of depth-slab maps (Section 2.1: the radiative transfer along a line of
 * sight applies the farther material first; Section 4.2.2: tasks render their particles
 * independently, here one depth slab each with SPLOTCH_OUT_MAP).  maps: device, n_maps
 * arrays of `pixels` x 6 FP32 one after the other, the farthest slab first, each pixel
 * holding (alpha_r, alpha_g, alpha_b, beta_r, beta_g, beta_b) of I_out = alpha I_in +
 * beta.  out: device, pixels x 6, the composed map: per pixel and channel, from the
 * farthest map on, beta <- alpha_k beta + beta_k (one rounding) and alpha <- alpha_k alpha;
 * its beta is the frame from a black background.  out must not overlap maps; the caller
 * owns both.  Asynchronous on `stream`.  Errors: INVALID_ARG (n_maps < 1, pixels < 0,
 * NULL buffers, overlap), CUDA. */
splotch_status splotch_compose_maps(const float *maps, int32_t n_maps, int64_t pixels, float *out, void *stream);

/* Test hook: per-particle raster outputs for one view, out8 = device float[8][n]:
 * X, Y, R, zc, e_r, e_g, e_b (emission = brightness x colour), active (0 / 1).
 * Inactive particles have X = Y = R = 0 when culled by the near plane. */
splotch_status splotch_debug_raster(splotch_scene *scene, const splotch_camera *cam,
                                    const splotch_render_params *params, float *out8,
                                    void *stream);

/* Test hook: tile lists of one view.  counts: device int32[n_tiles]; offsets: device
 * int64[n_tiles + 1]; members: device int32[capacity] particle indices, grouped by tile
 * in tile order (row-major), order inside a tile unspecified; *total (host) = pair
 * count.  Returns CAPACITY (with *total set) if capacity is too small.  Synchronous. */
splotch_status splotch_debug_bins(splotch_scene *scene, const splotch_camera *cam,
                                  const splotch_render_params *params, int32_t *counts,
                                  int64_t *offsets, int32_t *members, int64_t capacity,
                                  int64_t *total, void *stream);

/* Batched multi-view plan: all views share W x H and tile size.  Creation renders the
 * pair counts of `cams` once to size the tile lists (times `headroom` >= 1) and keeps
 * every buffer; splotch_plan_launch then enqueues the whole frame batch (count, scan,
 * scatter and one persistent splat launch over all views' work) with no host
 * synchronisation, so it may be captured into a CUDA graph.  If a launch needs more
 * pairs than were reserved, its kernels skip their work and splotch_plan_check reports
 * SPLOTCH_ERR_CAPACITY with the pairs needed; recreate the plan then. */
splotch_status splotch_plan_create(splotch_scene *scene, const splotch_camera *cams,
                                   int32_t n_views, const splotch_render_params *params,
                                   double headroom, void *stream, splotch_plan **out);

/* Replace the plan's cameras (same count and image size); stream-ordered copy. */
splotch_status splotch_plan_set_cameras(splotch_plan *plan, const splotch_camera *cams,
                                        int32_t n_views, void *stream);

/* Per-view brightness of a plan (Section 2.1: a scene file varies parameters such as the
 * brightness over a progression of images that make a movie).  scale: host,
 * n_views x n_types floats (view-major), each finite and >= 0: the emission of species t
 * in view v is multiplied by scale[v * n_types + t]; NULL resets every scale to 1.  The
 * next launch (or graph replay) renders with these scales.  Synchronises `stream`.
 * Errors: INVALID_ARG (NULL plan, a negative or non-finite scale), CUDA. */
splotch_status splotch_plan_set_brightness(splotch_plan *plan, const float *scale, void *stream);

/* Per-view colormaps of a plan (Section 2.1: a scene file varies parameters such as the
 * colour palette over a progression of images).  cmap_rgb: host, n_views x n_types
 * pointers (view-major), each to cmap_len[v * n_types + t] RGB triples (FP32, finite,
 * 2..2^20 entries): the colormap of species t in view v, times the scene's brightness of
 * t (a brightness sequence still applies on top); NULL resets every view to the scene's
 * colormaps.  Palette thresholds are colormaps whose entries below / above a threshold
 * repeat the end colours.  The next launch (or graph replay) renders with these
 * colormaps; a captured graph is captured again when the plan's colormap storage moves.
 * Stream-ordered on `stream`, which it synchronises.  Errors: INVALID_ARG (NULL plan, a
 * bad colormap), UNSUPPORTED (a scene with vector colour, whose emission is per
 * particle), OOM, CUDA. */
splotch_status splotch_plan_set_colormaps(splotch_plan *plan, const float *const *cmap_rgb,
                                          const int32_t *cmap_len, void *stream);

/* Enqueue one batch render into out (device, n_views x H x W x 3 FP32). */
splotch_status splotch_plan_launch(splotch_plan *plan, float *out, void *stream);

/* Synchronise `stream` and report the last launch: OK, CAPACITY (pairs_needed set), or
 * TIMEOUT.  pairs_needed may be NULL. */
splotch_status splotch_plan_check(splotch_plan *plan, void *stream, int64_t *pairs_needed);

/* Device bytes a plan holds (its workspace), and its tile size. */
splotch_status splotch_plan_info(const splotch_plan *plan, int64_t *device_bytes,
                                 int32_t *tile, int64_t *pair_capacity);

/* Release a plan (NULL accepted). */
splotch_status splotch_plan_destroy(splotch_plan *plan);

/* Workspace bytes one splotch_render of `pairs` particle-tile pairs needs at this size,
 * for admission control by HBM footprint. */
int64_t splotch_workspace_bytes(const splotch_scene *scene, int32_t width, int32_t height,
                                int32_t tile, int64_t pairs);

/* Two-phase render of one view, for callers that share the device and must know a
 * frame's memory before it is taken (a request server admitting work by HBM footprint).
 * The phases are those of splotch_render: the count pass of the binning (Section 3.2.1:
 * every particle's member tiles, counted per tile), then the lists and the splat.
 *   splotch_frame_fixed_bytes: device bytes the count phase allocates for this scene,
 *     camera and parameters (-1 on invalid arguments).  No GPU work.
 *   splotch_frame_prepare: allocates those bytes (the scene's allocator, stream-ordered
 *     on `stream`), runs raster + count + scan and waits for them; returns the frame,
 *     its fixed bytes, the exact bytes splotch_frame_render will allocate (*var_bytes:
 *     the frame's tile lists and split-tile scratch) and its particle-tile pairs.
 *   splotch_frame_render: allocates exactly *var_bytes, then scatter + splat + final
 *     transform into `out` (device, H x W x 3 FP32, or as params->flags ask), ordered
 *     after the prepare stream; asynchronous unless SPLOTCH_SYNC.  Once per frame.
 *   splotch_frame_destroy: releases both allocations, ordered on the stream last used;
 *     NULL is accepted.
 * The caller owns `out`; the frame owns its workspace.  Errors as splotch_render;
 * INVALID_ARG when a frame is rendered twice. */
typedef struct splotch_frame splotch_frame;
int64_t splotch_frame_fixed_bytes(const splotch_scene *scene, const splotch_camera *cam,
                                  const splotch_render_params *params);
splotch_status splotch_frame_prepare(splotch_scene *scene, const splotch_camera *cam,
                                     const splotch_render_params *params, void *stream, splotch_frame **frame,
                                     int64_t *fixed_bytes, int64_t *var_bytes, int64_t *pairs);
splotch_status splotch_frame_render(splotch_frame *frame, float *out, void *stream);
splotch_status splotch_frame_destroy(splotch_frame *frame);

/* Self-test of the bounded device wait every kernel uses: one CTA waits on a shared-memory
 * mbarrier that nothing completes, gives up after ~limit_cycles SM cycles (1e3..1e10) and
 * reports it.  Returns SPLOTCH_ERR_TIMEOUT when the wait ran out as designed, SPLOTCH_OK
 * if the barrier completed (it cannot), INVALID_ARG / CUDA otherwise.  Synchronous. */
splotch_status splotch_selftest_bounded_wait(int64_t limit_cycles, void *stream);

/* Kernel durations (ms) of this thread's last splotch_render made with SPLOTCH_TIMING:
 * ms[0] raster+count, ms[1] scan, ms[2] raster+scatter, ms[3] splat+final; and the
 * frame's particle-tile pairs, work items and split tiles in counts[0..2].
 * INVALID_ARG if no timed render has run on this thread. */
splotch_status splotch_last_timing(double ms[4], int64_t counts[3]);

/* Render one view without allocating any device memory.  The paper has no counterpart:
 * this serves callers that cannot allocate while they render (a host application that
 * owns all device memory through its own manager, a real-time loop that forbids
 * allocation after start-up, since an allocation can block on the device).  The frame
 * workspace lives in a fixed 32 MiB device array inside this library, present on every
 * GPU that loads the library until the process exits.  The caller passes the scene
 * (created earlier with splotch_create_scene, on the device that is current for this
 * call: INVALID_ARG otherwise), the camera, the parameters and `out` (device, H x W x 3
 * FP32), as for splotch_render.  The first call on a device looks up that device's copy
 * of the array; make it before any stream capture.  The call waits for the frame (it
 * synchronises `stream`).  All calls on a device share the array and each clears what it
 * counts into, so calls that overlap on the GPU (other threads, other streams) race and
 * must be serialised by the caller.
 * Limits: up to 2 MiB of per-chunk tile bases; up to 256 tiles split across work items,
 * whose exact accumulators (48 x T^2 bytes each) take at most 8 MiB (so 170 at 32-px
 * tiles, 42 at 64-px tiles); and the particle-tile records of the frame in the rest of
 * the 32 MiB (16 bytes each; about 1.5 million at 1024 tiles of 16 px).  Frames beyond
 * that return SPLOTCH_ERR_CAPACITY (the kernels skip the work; `out` is not written);
 * images whose tile tables do not fit return SPLOTCH_ERR_UNSUPPORTED before any GPU work.
 * Other errors as splotch_render. */
splotch_status splotch_render_noalloc(splotch_scene *scene, const splotch_camera *cam,
                                      const splotch_render_params *params, float *out, void *stream);

/* Test hook: stable sort of n (key, value) pairs on the device by key bits
 * [bit_lo, bit_hi) (a multiple of 8 bits), in place: the least-significant-digit radix
 * sort of the depth-ordered render (particles by depth, then records by tile).  keys:
 * device, n unsigned integers of key_bytes (4 or 8) bytes each; vals: device, n uint32;
 * n < 2^32.  Synchronous.  Errors: INVALID_ARG, UNSUPPORTED, OOM, CUDA. */
splotch_status splotch_debug_sort(void *keys, int32_t key_bytes, uint32_t *vals, int64_t n, int32_t bit_lo,
                                  int32_t bit_hi, void *stream);

/* Static strings. */
const char *splotch_status_string(splotch_status status);
const char *splotch_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* SPLOTCH_H */
