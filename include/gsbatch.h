/* gsbatch -- batched forward 3D Gaussian Splatting (RGB + depth) for many
 * environments on one GB300 (sm_103a).
 *
 * The problem statement follows the paper's simulation loop (Sec. III-A
 * "Data Flow"): a physics step yields rigid-body poses, Rigid-Link Gaussian
 * Kinematics (Sec. III-C "RLGK") moves the Gaussian clusters bound to each
 * rigid link, and the batch 3DGS renderer (Sec. III-C "Throughput Scaling",
 * built on the 3DGS forward pass the paper cites in Sec. II-B) returns RGB
 * images and depth maps for every environment.
 *
 * Conventions (the paper states none; these are the library's readings):
 *   world z up; camera axes x right, y down, z forward (OpenCV);
 *   a pose is a unit quaternion (w,x,y,z) then a translation;
 *   link poses map link -> world, camera poses map world -> camera;
 *   pixel (i,j) has its centre at (i+0.5, j+0.5);
 *   near plane per camera, 1.3 frustum guard band, 0.3 px^2 low-pass,
 *   alpha = min(0.99, o exp(-q/2)), alpha floor 1/255, stop when
 *   T (1 - alpha) < 1e-4, depth order ties broken by ascending global index
 *   (background 0..N_b-1 in the caller's order, then link Gaussians in
 *   link-major order),
 *   black background, rgb clamped to [0,1], depth = sum(alpha T z)/(1-T)
 *   (0 where 1-T = 0), SH colour max(0, sum sh_k Y_k(d) + 0.5) with the view
 *   direction d taken in the link frame for link Gaussians.
 *
 * Errors: every call returns a gs_status; no call throws, exits or traps.
 * gs_last_error() returns a thread-local message for the last failure.
 * Argument checks fail with GS_ERR_INVALID before anything is launched.
 * Faults found on the device (a zero or non-finite pose quaternion, a
 * capacity overflow) are recorded in the scene's device status word and
 * reported by gs_scene_sync_status().
 *
 * Threading: a gs_scene may be used from one host thread at a time.
 */
#ifndef GSBATCH_H
#define GSBATCH_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct gs_scene_s* gs_scene;

typedef enum {
    GS_OK = 0,
    GS_ERR_INVALID = -1,     /* bad argument; nothing was launched */
    GS_ERR_OOM = -2,         /* device allocation failed or the scratch budget is too small */
    GS_ERR_CUDA = -3,        /* a CUDA runtime call failed (message in gs_last_error) */
    GS_ERR_TIMEOUT = -4,     /* a bounded device wait gave up */
    GS_ERR_UNSUPPORTED = -5, /* valid request outside what the library implements */
    GS_ERR_DEVICE = -6       /* the device status word reports a fault (see gs_scene_sync_status) */
} gs_status;

typedef enum { GS_F32 = 0, GS_BF16 = 1, GS_F16 = 2 } gs_dtype;

/* A borrowed structure-of-arrays view of n Gaussians.  The library copies what
 * it needs during the call; the caller keeps ownership.
 *   mean      float32 [n][3]
 *   quat      float32 [n][4]  (w,x,y,z), need not be normalised, must be non-zero
 *   log_scale dtype   [n][3]  per-axis log standard deviation
 *   opacity   dtype   [n]     activated opacity in (0,1]
 *   sh        dtype   [n][sh_coeffs][3]  coefficient-major, channel-minor,
 *             coefficient k = l*l + l + m (3DGS order), sh_coeffs = (sh_degree+1)^2
 *   on_device non-zero if the pointers are device memory, else host memory.
 * dtype GS_BF16 / GS_F16 applies to log_scale, opacity and sh (the storage
 * form of the precision variant); mean and quat are always float32. */
typedef struct {
    int64_t n;
    const float* mean;
    const float* quat;
    const void* log_scale;
    const void* opacity;
    const void* sh;
    int sh_degree; /* 0..3 */
    gs_dtype dtype;
    int on_device;
} gs_gaussians;

/* One pinhole camera, world -> camera.  56 bytes, no padding. */
typedef struct {
    float fx, fy, cx, cy;
    int32_t width, height;
    float q_cw[4]; /* (w,x,y,z) */
    float t_cw[3];
    float near_plane; /* > 0; 0.01 m in the standard workloads */
} gs_camera;

/* Create a scene holding a static background (world-frame Gaussians, may be
 * empty: n = 0).  The scene owns device copies of the attributes in its own
 * layout (per-Gaussian 3D covariance derived from quat and log_scale, SH in
 * coefficient-plane-major order) and in its own order: the background is
 * stored in Morton (Z-order) order of the means within their bounding box (10
 * bits per axis; equal codes keep the caller's order), so that neighbouring
 * Gaussians, which mostly share their visibility, are projected together
 * (gs_scene_get_order gives it).  The order is internal: equal depths still
 * composite by the caller's global index, and every per-Gaussian output
 * (contribution scores, debug copies) is indexed by the caller's order.  Uses the current CUDA device; synchronises that
 * device.  Errors: GS_ERR_INVALID (null/negative/ill-formed view, zero
 * quaternion), GS_ERR_OOM, GS_ERR_CUDA. */
gs_status gs_scene_create(const gs_gaussians* background, gs_scene* out);

/* The background's storage order: order[k] (HOST int64 [n], n >= the
 * background's size) receives the caller's index of the background Gaussian
 * stored at position k.  Nothing is written for an empty background.
 * Errors: GS_ERR_INVALID (null scene, null or short order). */
gs_status gs_scene_get_order(gs_scene s, int64_t* order, int64_t n);

/* Bind link-frame Gaussian clusters to n_links rigid links (RLGK, Sec. III-C):
 * link l owns link_gaussians[link_offsets[l] .. link_offsets[l+1]) (host array
 * of n_links+1 non-decreasing offsets, link_offsets[0] = 0,
 * link_offsets[n_links] = link_gaussians->n).  Replaces any earlier links.
 * The dtype and sh_degree must equal the background's (if it is non-empty).
 * Errors as gs_scene_create. */
gs_status gs_scene_attach_links(gs_scene s, int n_links, const int64_t* link_offsets,
                                const gs_gaussians* link_gaussians);

/* Render n_envs environments of one resolution (all cams[e].width/height equal).
 *   link_poses  DEVICE float32 [n_envs][n_links][7], (qw,qx,qy,qz,tx,ty,tz), link -> world
 *               (may be NULL when n_links = 0)
 *   cams        HOST   gs_camera [n_envs]
 *   rgb         DEVICE float32 [n_envs][H][W][3]
 *   depth       DEVICE float32 [n_envs][H][W]
 *   alpha       DEVICE float32 [n_envs][H][W] or NULL
 *   cuda_stream cudaStream_t (NULL = legacy default stream)
 * All launches are ordered on cuda_stream.  The call blocks the host once per
 * wave of environments for a 16-byte read of the intersection total (to size
 * the scratch), so it returns after the last wave's launches are queued, not
 * after they finish.  Scratch memory is owned by the scene, grown on demand
 * up to the budget (gs_scene_set_budget).  n_envs = 0 is a no-op.
 * Errors: GS_ERR_INVALID (bad pointers or camera parameters), GS_ERR_OOM,
 * GS_ERR_CUDA; device-side faults via gs_scene_sync_status. */
gs_status gs_render_batch(gs_scene s, int n_envs, const float* link_poses, const gs_camera* cams, float* rgb,
                          float* depth, float* alpha, void* cuda_stream);

/* As gs_render_batch, but link_poses, rgb, depth and alpha are HOST buffers.
 * The library copies the poses in.  Page-locked outputs (cudaHostAlloc /
 * cudaMallocHost / registered memory) are mapped into the device's address
 * space, so the compositor stores the images straight into them; other host
 * memory is rendered wave by wave into device staging and each wave's images
 * are copied out while the next wave renders.  The call returns when all
 * images are on the host. */
gs_status gs_render_batch_host(gs_scene s, int n_envs, const float* link_poses, const gs_camera* cams, float* rgb,
                               float* depth, float* alpha, void* cuda_stream);

/* Observation form.  Policies consume 8-bit images; the paper's manipulation
 * experiments randomise image-level appearance (brightness, contrast and
 * exposure) during training (Sec. IV-E).  The library applies both in the
 * compositor's store, per environment:
 *   c  = clamp(colour, 0, 1) per channel (the float image's value)
 *   v  = clamp((c * 2^exposure - 0.5) * contrast + 0.5 + brightness, 0, 1)
 *   u8 = round-to-nearest-even(255 v)
 * in FP32 with fused multiply-adds; depth (the float image's value) is
 * rounded to IEEE half.  {exposure 0, contrast 1, brightness 0} leaves the
 * colour unchanged.  12 bytes. */
typedef struct {
    float exposure;    /* stops: linear gain 2^exposure */
    float contrast;    /* scale about 0.5 */
    float brightness;  /* offset */
} gs_appearance;

/* As gs_render_batch, writing the observation form:
 *   appearance  DEVICE gs_appearance [n_envs], or NULL for the identity
 *   rgb8        DEVICE uint8 [n_envs][H][W][3]
 *   depth16     DEVICE uint16 (half bits) [n_envs][H][W], or NULL (no depth)
 * 4 (RGB) + 2 (depth) bytes per pixel instead of 16.  Errors as
 * gs_render_batch. */
gs_status gs_render_batch_obs(gs_scene s, int n_envs, const float* link_poses, const gs_camera* cams,
                              const gs_appearance* appearance, uint8_t* rgb8, uint16_t* depth16, void* cuda_stream);

/* As gs_render_batch_obs with HOST link_poses, appearance, rgb8 and depth16
 * (copied in and out as in gs_render_batch_host); returns when the images are
 * on the host. */
gs_status gs_render_batch_obs_host(gs_scene s, int n_envs, const float* link_poses, const gs_camera* cams,
                                   const gs_appearance* appearance, uint8_t* rgb8, uint16_t* depth16,
                                   void* cuda_stream);

/* Batch-LiDAR (the paper's ray-casting LiDAR over the same Gaussians, with
 * dynamic objects and self-occlusion, Sec. III-E and Table II).  A LiDAR of
 * `rows` beams x `cols` azimuth steps over the azimuth window [az_min,
 * az_max): a rotating LiDAR covers a full revolution (0, 2 pi), a solid-state
 * one a narrower field of view; sensor frame x forward, y left, z up; ray
 * (i, j) has azimuth az_min + (az_max - az_min) (i + 1/2) / cols and
 * elevation elev_min + (elev_max - elev_min) (j + 1/2) / rows.  Each ray is composited
 * front to back like a camera pixel (alpha = min(0.99, o exp(-q/2)) >= 1/255,
 * stop when T (1 - alpha) < 1e-4, order by distance of the Gaussian's centre
 * from the sensor, ties by global index), the Gaussian evaluated at its
 * closest approach along the ray: with G = diag(e^-s) R^T in the sensor
 * frame, a = G d and b = G mu, q = |a x b|^2 / |a|^2 at t* = a.b / |a|^2;
 * Gaussians with t* <= near_range are skipped.  56 bytes. */
typedef struct {
    float q_ws[4];     /* world -> sensor rotation (w,x,y,z) */
    float t_ws[3];     /* world -> sensor translation */
    int32_t rows;      /* beams */
    int32_t cols;      /* azimuth steps across the window */
    float elev_min;    /* radians */
    float elev_max;    /* radians, > elev_min, both within (-pi/2, pi/2) */
    float near_range;  /* > 0 */
    float az_min;      /* radians, finite */
    float az_max;      /* radians, az_min < az_max <= az_min + 2 pi */
} gs_lidar;

/* Scan n_envs environments:
 *   link_poses  DEVICE as for gs_render_batch
 *   sensors     HOST gs_lidar [n_envs] (all with the same rows and cols)
 *   range       DEVICE float32 [n_envs][rows][cols]: sum(alpha T t*) / (1 - T), 0 where nothing is hit
 *   hit         DEVICE float32 [n_envs][rows][cols] (1 - T), or NULL
 * Bins on 16x16 tiles of the (azimuth, beam) grid whatever the scene's tile
 * setting.  Errors as gs_render_batch (GS_ERR_INVALID for a bad sensor). */
gs_status gs_render_lidar(gs_scene s, int n_envs, const float* link_poses, const gs_lidar* sensors, float* range,
                          float* hit, void* cuda_stream);

/* Scan n_envs environments along arbitrary rays: the non-repetitive scan
 * patterns of the paper's LiDAR list (Sec. III-E, Table II), whose rays are
 * not a regular (azimuth, beam) grid.  Each ray is composited exactly as a
 * ray of gs_render_lidar.
 *   sensors   HOST gs_lidar [n_envs]: pose and near_range as for
 *             gs_render_lidar; rows, cols, elevation range and azimuth window
 *             only describe a binning grid (all sensors alike) that must
 *             contain every ray direction: a zero direction, or one outside
 *             the grid, reads 0 and sets the device status word
 *             (gs_scene_sync_status reports it).  About one ray per cell bins
 *             best; any density is correct.
 *   n_rays    rays per environment, 1 .. 2^24
 *   ray_dirs  DEVICE float32 [n_envs][n_rays][3]: directions in the sensor
 *             frame (x forward, y left, z up; need not be unit length)
 *   range     DEVICE float32 [n_envs][n_rays]: sum(alpha T t*) / (1 - T), 0 where nothing is hit
 *   hit       DEVICE float32 [n_envs][n_rays] (1 - T), or NULL
 * Blocks the host once per wave (intersection and ray totals).  Errors as
 * gs_render_lidar (GS_ERR_INVALID also for n_rays out of range or a null
 * ray_dirs). */
gs_status gs_render_rays(gs_scene s, int n_envs, const float* link_poses, const gs_lidar* sensors, int n_rays,
                         const float* ray_dirs, float* range, float* hit, void* cuda_stream);

/* Contribution pass (support for pruning, a scene transform that follows the
 * paper's Gaussian pruning for speed and memory, Sec. III-C): renders n_envs
 * environments like gs_render_batch (one resolution, 16x16 tiles whatever
 * the scene's tile setting) without writing images, and ADDS to scores[g],
 * for every Gaussian g, the sum over pixels of its blending weight alpha T
 * where it was composited.  scores: DEVICE float [background + link
 * Gaussians], the caller's order; the caller zeroes it.  Sum over g of the added
 * weights = sum over pixels of alpha (the weights telescope).  Errors as
 * gs_render_batch. */
gs_status gs_scene_contribution(gs_scene s, int n_envs, const float* link_poses, const gs_camera* cams,
                                float* scores, void* cuda_stream);

/* Pruning as a scene transform (the paper prunes Gaussians for speed and
 * memory, Sec. III-C, keeping about 30 % of a static scene and up to 90 %
 * fewer on dynamic objects; it does not give its criterion).  Ranks the
 * Gaussians by score, descending (equal scores: lower index first), and
 * creates a new scene (*out, destroyed by the caller) holding the top
 * ceil(keep_bg n_bg) background Gaussians and the top ceil(keep_links n_l) of
 * every link's cluster, kept in their original order: the new scene's
 * background index and link offsets number the kept Gaussians in the caller's
 * order, and they render exactly as in the source scene.  The source scene is
 * unchanged.
 *   scores     DEVICE float32 [background + link Gaussians], the caller's order
 *              (for instance gs_scene_contribution's weights); no NaN
 *   keep_bg, keep_links  fractions in [0, 1]
 *   kept       HOST int64 [kept_cap] or NULL: receives, for every Gaussian of
 *              the new scene (background, then link-major), its index in the source
 * Selection and the new scene's attributes are computed on the device; the
 * call synchronises it.  Errors: GS_ERR_INVALID (null handle or scores,
 * fraction out of range, NaN score, kept_cap below the kept count),
 * GS_ERR_OOM, GS_ERR_CUDA. */
gs_status gs_scene_prune(gs_scene s, const float* scores, double keep_bg, double keep_links, gs_scene* out,
                         int64_t* kept, int64_t kept_cap);

/* One environment of an uneven batch (gs_render_batch_v, plans).  80 bytes. */
typedef struct {
    gs_camera cam;        /* its own camera, width and height */
    int32_t link_begin;   /* renders the scene's links [link_begin, link_end) on top of the background */
    int32_t link_end;
    int64_t pose_offset;  /* index, in units of 7 floats, of the pose of link_begin in link_poses */
    int64_t pixel_offset; /* first pixel of this env's image: rgb[3*pixel_offset..], depth[pixel_offset..] */
} gs_env;

/* Render environments of different resolutions and link subsets in one call
 * (the batched uneven form; each env's (env, tile) work items run in the same
 * persistent compositing launch).  envs: HOST array; link_poses, rgb, depth,
 * alpha: DEVICE.  Images may be placed anywhere in the output buffers through
 * pixel_offset (they must not overlap).  Results equal gs_render_batch for
 * the same env.  Tile shape, budget and waves as for gs_render_batch.
 * Errors: GS_ERR_INVALID (bad camera, link range outside the scene, negative
 * offsets), GS_ERR_OOM, GS_ERR_CUDA. */
gs_status gs_render_batch_v(gs_scene s, int n_envs, const gs_env* envs, const float* link_poses, float* rgb,
                            float* depth, float* alpha, void* cuda_stream);

/* A plan is a fixed batch (environments, resolutions, link subsets) rendered
 * repeatedly with changing poses.  Its first launch runs eagerly: with
 * GS_PLAN_AUTOTUNE it times every tile shape (8x8, 16x8, 16x16, 32x8, 32x16) and
 * compositor claim size (1 or 4 tiles per atomic), on 16x16 and 8x8 tiles also
 * the compositor's quadrant form (lanes in groups of eight, each group walking
 * the splats of its own 4x4 pixel quadrant), and keeps the fastest (the
 * images do not depend on the choice); it sizes the intersection-key buffer at
 * 1.25x what that launch needed.  With GS_PLAN_GRAPH the whole render (all
 * waves) is then captured in a CUDA graph and later launches replay it with
 * no host synchronisation (re-captured when the pose or output pointers
 * change).  If poses later need more keys than the capacity, the extra keys
 * are dropped, the scene's status word reports it (gs_scene_sync_status), and
 * the next launch after that one completed re-measures the need with an eager
 * pass (host-synchronising), resizes to 1.25x and re-captures.  The plan owns
 * its scratch (separate from the scene's). */
enum { GS_PLAN_AUTOTUNE = 1, GS_PLAN_GRAPH = 2 };
typedef struct gs_plan_s* gs_plan;
typedef struct {
    int tile_w, tile_h;     /* chosen tile shape */
    int chunk;              /* chosen compositor claim size */
    int waves;              /* waves per launch */
    int graph;              /* 1 once a CUDA graph is instantiated */
    int tuned_candidates;   /* configurations timed by the autotuner */
    double tuned_ms;        /* eager time of the chosen configuration */
    int regrows;            /* capacity re-measurements after overflows */
    int64_t key_capacity;   /* intersection keys, all waves */
    int64_t scratch_bytes;  /* device scratch held by the plan */
    int quad;               /* 1 if the compositor runs its quadrant form (16x16 or 8x8 tiles) */
} gs_plan_info;
gs_status gs_plan_create(gs_scene s, int n_envs, const gs_env* envs, int flags, gs_plan* out);
gs_status gs_plan_launch(gs_plan p, const float* link_poses, float* rgb, float* depth, float* alpha,
                         void* cuda_stream);
gs_status gs_plan_get_info(gs_plan p, gs_plan_info* out);
void gs_plan_destroy(gs_plan p);

/* As gs_render_batch (same arguments, same kernels, same results), but it
 * allocates nothing: no cudaMalloc, cudaFree or allocating library call.  The
 * paper has no counterpart; this is for callers that must not allocate device
 * memory while rendering -- a process whose GPU memory is already reserved by
 * another allocator, code running where an allocation would stall the device
 * (cudaFree synchronises it) or is not allowed, a control loop that cannot
 * absorb a first-time allocation.
 * Its working memory is one file-scope device array of 32 MiB per device,
 * held by every process that loads the library until it exits.  The first
 * call on a device looks up that array's device address (once per device,
 * with the device current); make that first call before any stream capture.
 * Every call on a device shares the array and it keeps the last call's data:
 * each call clears the counters it needs zeroed, and calls whose work
 * overlaps on the GPU (other streams or threads) race on it.
 * Sizes beyond the array fail with GS_ERR_UNSUPPORTED and a message giving the
 * bytes needed: before any launch when one environment's projected records
 * do not fit, or after the binning of a wave when its intersection keys do
 * not fit (earlier waves' images are then complete, later ones unwritten).
 * Like gs_render_batch it reads one wave total back to the host per wave of
 * up to 256 environments (into a stack buffer): each wave waits on
 * cuda_stream once (cudaStreamSynchronize), so the call returns after the
 * last wave's launches are queued.  Calls are serialised on the host: one
 * lock guards the static host tables of the waves for the whole call, so
 * concurrent calls from other threads wait, even for other devices. */
gs_status gs_render_batch_noalloc(gs_scene s, int n_envs, const float* link_poses, const gs_camera* cams,
                                  float* rgb, float* depth, float* alpha, void* cuda_stream);

/* Tile shape used by the binning and compositing kernels.  Allowed:
 * 8x8, 16x8, 16x16, 32x8, 32x16 (tw x th).  Results do not depend on the tile shape
 * (each splat's support box is inflated by a relative 1e-4 so every tile it
 * may reach sees it).  Default 16x16. */
gs_status gs_scene_set_tile(gs_scene s, int tile_w, int tile_h);

/* Upper bound, in bytes, on the scene's device scratch (records, masks,
 * intersection lists).  Environments are rendered in waves sized to fit.
 * Default 64 GiB.  GS_ERR_OOM from gs_render_batch if one env does not fit. */
gs_status gs_scene_set_budget(gs_scene s, int64_t bytes);

/* Maximum environments per wave (0 = as many as the budget allows). */
gs_status gs_scene_set_wave(gs_scene s, int max_envs_per_wave);

/* Wait for the scene's work on cuda_stream, then read and clear the device
 * status word.  GS_OK, or GS_ERR_DEVICE with a description in gs_last_error. */
gs_status gs_scene_sync_status(gs_scene s, void* cuda_stream);

/* Counters of the last gs_render_batch call (host-side values; the pair total
 * is the sum over waves of the intersection totals read during the call). */
typedef struct {
    int64_t waves;          /* waves rendered */
    int64_t kernel_launches;/* kernels launched by the call */
    int64_t intersections;  /* (env, tile) intersections, all waves */
    int64_t scratch_bytes;  /* device scratch currently held by the scene */
    int64_t n_gaussians;    /* background + link Gaussians */
    int64_t composited;     /* with counters on: (pixel, Gaussian) pairs with alpha >= 1/255
                               examined before termination, summed since counters were enabled */
    int64_t visible;        /* with counters on: (env, Gaussian) pairs projected to a record
                               (non-empty support on screen), summed since counters were enabled */
    int64_t fp64_conics;    /* with counters on: (env, Gaussian) pairs whose 2D covariance was near
                               degenerate (AC - B^2 < 2^-10 AC before the low-pass) and was inverted
                               in FP64, summed since counters were enabled */
} gs_stats;
/* Synchronises the device when counters are on (to read the device counter). */
gs_status gs_scene_get_stats(gs_scene s, gs_stats* out);

/* Count composited (pixel, Gaussian) pairs in the compositor (adds one shared
 * reduction and one atomic per tile; off by default).  Enabling resets the count. */
gs_status gs_scene_set_counters(gs_scene s, int enable);

/* Per-kernel device time.  With profiling on, every launch of a render is
 * bracketed by CUDA events recorded on the render's stream; gs_scene_get_timings
 * waits for the recorded events and returns milliseconds and launch counts per
 * phase, accumulated since the last reset. */
enum {
    GS_PHASE_LINK = 0,      /* A1: link composition */
    GS_PHASE_PROJECT = 1,   /* A2: projection + SH */
    GS_PHASE_COUNT = 2,     /* A3: intersection counting */
    GS_PHASE_SCAN = 3,      /* A3: prefix scans */
    GS_PHASE_SCATTER = 4,   /* A4: bucketed key scatter */
    GS_PHASE_COMPOSITE = 5, /* A4 sort + A5 compositing */
    GS_PHASES = 6
};
typedef struct {
    double ms[GS_PHASES];
    int64_t launches[GS_PHASES];
} gs_timings;
gs_status gs_scene_set_profile(gs_scene s, int enable);
gs_status gs_scene_get_timings(gs_scene s, gs_timings* out, int reset);

/* Debug hooks for parity tests.  When enabled, the next gs_render_batch
 * keeps, for the env of the LAST wave given by gs_debug_copy_* (local index
 * within that wave), the projected records and the depth-sorted per-tile
 * lists, in addition to its normal outputs (slower; off by default). */
gs_status gs_scene_set_debug(gs_scene s, int enable);

/* Copy env `env` (absolute index, must belong to the last wave rendered) of
 * the projected records to HOST arrays of n = background + link Gaussians:
 *   visible u8 [n]; u, v, hx, hy, z, opacity f32 [n]; conic f32 [n][3];
 *   rgb f32 [n][3]; range i32 [n][4] (i0,i1,j0,j1).
 * Entries of invisible Gaussians are left as they were.  Synchronises. */
gs_status gs_debug_copy_records(gs_scene s, int env, uint8_t* visible, float* u, float* v, float* hx, float* hy,
                                float* z, float* opacity, float* conic, float* rgb, int32_t* range);

/* Copy env `env`'s per-tile intersection counts (u32 [tiles], row-major tile
 * grid) and, if lists is non-NULL, the depth-ordered per-tile lists of global
 * indices in the caller's order (u32 [sum counts], tiles in order).  Lists are available only when
 * debug was enabled for that render.  Synchronises. */
gs_status gs_debug_copy_tiles(gs_scene s, int env, uint32_t* counts, int64_t n_counts, uint32_t* lists,
                              int64_t n_lists);

/* Destroy a scene and free its device memory (NULL is a no-op). */
void gs_scene_destroy(gs_scene s);

/* ------------------------------------------------------------------ serving
 * A request loop over resident scenes.  The paper renders RGB-D for every
 * environment as the simulator steps (Sec. III-A, Sec. III-C); here envs step at
 * their own pace, each step is a render request, and a scheduler thread in
 * the library batches them continuously:
 *   - scenes (gs_scene, attached links) and per-env state (camera, link
 *     range, the RGB and depth images) stay resident on the device;
 *   - a request carries the env's link poses (host, copied at submit) and an
 *     arrival time; requests that have arrived are admitted, oldest first,
 *     into batches of one scene whose envs are idle (an env has at most one
 *     request in flight, so its results come back in submission order);
 *   - a batch is admitted when a stream slot is free and its estimated
 *     device working set (records, tile tables and intersection keys, the
 *     keys estimated from earlier batches of the same scene and resolution)
 *     fits the HBM budget beside the batches in flight; one batch holds at
 *     most budget / max_inflight (each slot keeps its scratch, so all slots
 *     together stay within the budget); a request that alone exceeds the
 *     budget still runs, alone, when nothing else is in flight;
 *   - each batch runs the full render on its own CUDA stream and scratch, so
 *     batches overlap on the device; a host callback on the stream records
 *     its completion time.  Its intersection keys get a capacity from the
 *     running per-(scene, resolution) estimate, so the scheduler never waits
 *     on the device; a batch whose keys overflowed it (flagged on the device)
 *     is rendered again with exact sizing before it completes, and the first
 *     batch of each kind is sized exactly;
 * A request's output is bit-identical to rendering its env alone with
 * gs_render_batch_v at the server's tile shape.  While a server runs, its
 * scenes must not be rendered or destroyed by other calls.
 * Times are seconds since gs_server_start (steady clock). */
typedef struct gs_server_s* gs_server;

typedef struct {
    int64_t budget_bytes;  /* device working-set budget of the batches in flight (>= 1 MiB) */
    int max_inflight;      /* stream slots, 1..64 */
    int max_batch_envs;    /* requests per batch, >= 1 */
    int tile_w, tile_h;    /* tile shape: 8x8, 16x8, 16x16, 32x8 or 32x16 */
} gs_server_config;

typedef struct {
    int64_t request_id;
    int env_id;
    int status;            /* 0 done; 1 cancelled; a negative gs_status on failure */
    double arrival_s;      /* scheduled arrival */
    double admit_s;        /* admitted into a batch (-1 if never) */
    double done_s;         /* completed on the device (host callback), or cancelled */
} gs_request_result;

typedef struct {
    int64_t submitted, completed, cancelled, batches;
    int64_t peak_inflight_bytes;  /* largest estimated working set in flight */
    int32_t max_concurrent;       /* most batches in flight at once */
    int32_t max_batch;            /* most requests in one batch */
    int64_t retried;              /* batches rendered again after their keys overflowed the estimate */
} gs_server_stats;

/* Create a server on the current device (stream slots created here; scratch
 * grows on first use).  GS_ERR_INVALID for a bad config. */
gs_status gs_server_create(const gs_server_config* cfg, gs_server* out);
/* Register a scene (borrowed; must outlive the server).  Before start only. */
gs_status gs_server_add_scene(gs_server sv, gs_scene scene, int* scene_id);
/* Register an env instance of a scene: camera (copied), links [link_begin,
 * link_end) of the scene.  Before start only. */
gs_status gs_server_add_env(gs_server sv, int scene_id, const gs_camera* cam, int link_begin, int link_end,
                            int* env_id);
/* Allocate the resident outputs and start the scheduler thread. */
gs_status gs_server_start(gs_server sv);
/* Submit a render request for env_id: link_poses host f32 [link_end -
 * link_begin][7] (copied; may be NULL for an env without links), arrival in
 * seconds since start (< 0: now).  Requests may be submitted before start
 * (open-loop arrival schedules).  request_id may be NULL. */
gs_status gs_server_submit(gs_server sv, int env_id, const float* link_poses, double arrival_s,
                           int64_t* request_id);
/* Cancel a request that has not been admitted yet: it completes with status 1.
 * GS_ERR_INVALID if it is unknown, admitted or finished. */
gs_status gs_server_cancel(gs_server sv, int64_t request_id);
/* Take up to max_results finished requests (completion order). */
gs_status gs_server_poll(gs_server sv, gs_request_result* out, int max_results, int* n_out);
/* Wait until every submitted request has finished (GS_ERR_TIMEOUT after
 * timeout_s), then read the scenes' device status words (GS_ERR_DEVICE as
 * gs_scene_sync_status).  A failed batch's CUDA error is returned here. */
gs_status gs_server_drain(gs_server sv, double timeout_s);
gs_status gs_server_get_stats(gs_server sv, gs_server_stats* out);
/* Seconds since gs_server_start (0 before start, -1 for NULL): the clock of
 * arrival_s, for scheduling arrivals relative to now. */
double gs_server_now(gs_server sv);
/* Device pointers to env_id's resident outputs: rgb f32 [H][W][3], depth f32
 * [H][W] (owned by the server; valid until destroy).  After start only; read
 * them when the env has no request in flight. */
gs_status gs_server_env_output(gs_server sv, int env_id, float** rgb, float** depth);
/* Stop the scheduler (requests not yet admitted are dropped), wait for the
 * batches in flight and free everything the server owns (NULL is a no-op). */
void gs_server_destroy(gs_server sv);

/* Measurement support (no paper counterpart): the current device's plain-ALU
 * rates, from two short microbenchmarks on cuda_stream (synchronises it):
 * FP32 FMA lane-ops/s (independent fmaf chains) and MUFU ex2 lane-ops/s
 * (ex2.approx chains), each the best of three timed runs after a warm-up.
 * The compositor is bound by these two pipes.  GS_ERR_CUDA on failure. */
gs_status gs_measure_alu_peak(double* fma_lane_ops_per_s, double* ex2_lane_ops_per_s, void* cuda_stream);

/* Thread-local description of the last failure ("" if none). */
const char* gs_last_error(void);

/* Library version string. */
const char* gs_version(void);

#ifdef __cplusplus
}
#endif

#endif /* GSBATCH_H */
