/* hdof -- hybrid ray-traced / post-processed depth of field on one GPU.
 *
 * C ABI of the per-frame hot path of "Hybrid DoF: Ray-Traced and
 * Post-Processed Hybrid Depth of Field Effect for Real-Time Rendering"
 * (Tan, Chua, Biette, Bhojan; SIGGRAPH '20 Posters).  The paper's pipeline
 * (Design section): a G-buffer with a sharp image, a post-process CoC filter
 * of that image, an adaptive ray mask, thin-lens distributed ray tracing of
 * the masked pixels, spatio-temporal reconstruction, and a composite.
 *
 * Conventions shared by every call
 * --------------------------------
 * - Pointers to image planes and scene arrays are DEVICE pointers owned by
 *   the caller.  Planes are row-major [height][width][channels], densely
 *   packed (pitch = width), pixel (i, j) = column i, row j from the top.
 * - Opaque handles (hdof_bvh) are owned by the library: create/destroy pairs.
 * - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).
 *   Every compute call only enqueues work and returns; results are ready
 *   when the stream reaches that point.
 * - Return value: HDOF_OK (0) or a negative HDOF_E* code.  Arguments are
 *   validated on the host before anything is enqueued (HDOF_EINVAL).  A
 *   launch failure returns HDOF_ECUDA.  hdof_last_error() gives the
 *   message of the calling thread's last failure.  Calls never throw.
 * - Kernel-side watchdogs (a capped traversal loop) never hang: they record
 *   HDOF_ETIMEOUT in a device status word that hdof_sync() reports.
 * - The library keeps per-device state for the life of the process (the
 *   post-filter's area table, the device addresses of its status word and of
 *   hdof_mask_noalloc's tile array): do not keep using it across a
 *   cudaDeviceReset of a device it has run on.
 * - The first post-filter call on a device (hdof_postfilter, the batched
 *   frame, hdof_post_forward/backward and their _dlens forms) uploads the
 *   area table and waits for it; make that first call before capturing a
 *   stream into a graph.
 * - Camera space: the camera at `pos` looks along +fwd with +right, +up;
 *   the screen point of pixel (i, j) this frame is (i + 0.5 + jitter[0],
 *   j + 0.5 + jitter[1]).  Depth is view-space z (distance along fwd).
 */
#ifndef HDOF_H
#define HDOF_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define HDOF_OK 0
#define HDOF_EINVAL (-1)
#define HDOF_ECUDA (-2)
#define HDOF_ENOMEM (-3)
#define HDOF_ETIMEOUT (-4)
#define HDOF_EUNSUPPORTED (-5)

/* storage types of the G-buffer planes */
#define HDOF_F32 0
#define HDOF_F16 1  /* nd: four halves (nx, ny, nz, z) */
#define HDOF_BF16 2 /* col: four bfloat16 (r, g, b, luminance) */

/* Pinhole camera of the frame (Design: the G-buffer is rendered with it;
 * Ray Trace: the thin-lens rays share its pose). */
typedef struct hdof_camera {
    float pos[3], right[3], up[3], fwd[3];
    float tan_half_fovy;
    int32_t width, height;
    float jitter[2];
} hdof_camera;

/* Thin lens (Potmesil and Chakravarty, cited in the Design section):
 * focus distance = view depth of the focus plane; aperture radius in scene
 * units.  CoC diameter in pixels: c(z) = A H (zf - z) / (z zf tan(fovy/2)),
 * positive in the near field.  focal_length is recorded, not used (it
 * cancels at fixed field of view). */
typedef struct hdof_lens {
    float focus_dist, aperture_radius, focal_length;
} hdof_lens;

/* Every constant of the method.  The paper prints none; each field is a
 * stated reading of its prose (see the per-call comments). */
typedef struct hdof_params {
    /* adaptive ray mask (Ray Trace section) */
    float gauss_sigma;   /* Gaussian 5x5 sigma on (n, z) */
    float edge_tau;      /* edge threshold on max(|grad n|, |grad z|/z) */
    int32_t tile;        /* mask tile edge in pixels */
    int32_t dilate;      /* tile dilation radius (tiles) */
    int32_t spp_max;     /* rays per edge-tile pixel, 1..255 */
    int32_t variance_on; /* add the temporal variance term */
    float var_tau;       /* luminance std-dev that keeps a pixel traced */
    float var_scale;     /* std-dev that earns spp_max rays */
    int32_t hlen_young;  /* history length below which a pixel gets spp_max */
    /* thin-lens ray trace (Ray Trace section) */
    uint32_t seed;       /* Philox key word 0 */
    int32_t frame, view; /* Philox key word 1 = view * 65536 + frame */
    float k_ambient;
    int32_t n_lights;    /* directional lights, 0..4 */
    float light_dir[4][3]; /* unit vectors towards the lights */
    float light_E[4];
    float miss_dist;     /* far position of a ray that hits nothing */
    int32_t trav_cap;    /* traversal step watchdog; 0 = default (64 x nodes) */
    /* temporal reconstruction (Reconstruction section) */
    float ema_alpha;
    int32_t camera_moved; /* compose with this frame's hit ratio */
    /* spatial reconstruction */
    float r_s;           /* gather radius cap, pixels */
    float var_ref;       /* std-dev at which the spatial gather is fully used */
    /* post-filter (Design section) */
    float r_max;         /* CoC radius cap, pixels, <= 100 */
    float kz_rel;        /* relative depth band of the far-field depth test */
    /* composite (Composite section) */
    float h_tau;         /* hit ratio above which far pixels take the post-process */
    /* extensions the paper's Discussion names as future work; 0 = off */
    float alpha_k;       /* per-pixel temporal blend factor: luminance change beyond alpha_k
                            history std-devs raises the pixel's EMA weight towards 1 */
    int32_t mask_coc;    /* 1: an edge tile's dilation reaches its pixels' largest CoC radius */
    int32_t blades;      /* aperture: 0 = circle, 3..16 = regular polygon of that many blades */
    float blade_rot;     /* polygon rotation, radians */
    float aberration;    /* lens sample weight 1 + aberration (2 rho^2 / A^2 - 1), in [-1, 1] */
    float spec_pref;     /* near branch: post-process share per unit of its specular intensity (Composite) */
} hdof_params;

/* G-buffer of one frame.  nd: (nx, ny, nz, z) per pixel, n the geometric
 * normal facing the viewer, z view depth (misses: z = miss_dist, n = -fwd);
 * col: (r, g, b, S) sharp shaded colour and its specular part S (the
 * highlight's luminance, 0 for Lambertian materials); mv: float2 motion (i, j)
 * minus the previous-frame index-space position of the surface point
 * (1e6 when the previous camera cannot see it); tri: original id of the hit
 * triangle, -1 for a miss.  mv and tri may be NULL for calls that do not
 * read them. */
typedef struct hdof_gbuf {
    int32_t width, height;
    int32_t dtype_nd;  /* HDOF_F32 (float4) or HDOF_F16 (half x4) */
    int32_t dtype_col; /* HDOF_F32 (float4) or HDOF_BF16 (bfloat16 x4) */
    void* nd;
    void* col;
    float* mv;
    int32_t* tri;
} hdof_gbuf;

/* Accumulated temporal history (one buffer per frame parity; a frame reads
 * the previous buffer and writes the other).  near = (EMA of h*C_near rgb,
 * EMA of h), far = (EMA of (1-h)*C_far rgb, EMA of 1-h), mom = (EMA of Y,
 * EMA of Y^2), hlen = frames accumulated (0 = no history).  All float32
 * except hlen (uint8).  Pixels with hlen = 0 hold don't-care values. */
typedef struct hdof_history {
    float* near_acc; /* [H][W][4] */
    float* far_acc;  /* [H][W][4] */
    float* mom;      /* [H][W][2] */
    uint8_t* hlen;   /* [H][W] */
} hdof_history;

typedef struct hdof_bvh hdof_bvh;

typedef struct hdof_bvh_stats {
    int32_t n_tris;
    int32_t n_nodes;  /* internal nodes */
    int32_t depth;    /* deepest leaf (bounds the traversal stack) */
    int32_t n_big;    /* scene-sized triangles tested outside the tree */
    int64_t device_bytes;
} hdof_bvh_stats;

/* ---------------------------------------------------------------- misc -- */
const char* hdof_version(void);
/* Copies the calling thread's last error message; returns its length. */
int hdof_last_error(char* buf, size_t n);
/* Synchronises `stream`, then reports (and clears) the device status word:
 * HDOF_ETIMEOUT if a kernel watchdog fired since the last call, HDOF_ECUDA
 * on a CUDA error, else HDOF_OK. */
int hdof_sync(void* stream);
/* Fills *p with the library defaults (the tiny-scene values). */
void hdof_default_params(hdof_params* p);

/* Kernel timing (not in the paper; a measurement facility).  With
 * hdof_profile(1) every compute call records a pair of CUDA events on its
 * stream around each of its kernels (names: "gbuffer", "mask",
 * "trace_compact", "trace_packets" or "trace_rays", "trace_resolve",
 * "pf_prep", "pf_rowscan", "pf_gather", "temporal", "spatial", "composite",
 * and the batched forms with a "batch_" prefix); hdof_profile(0) stops.
 * Do not profile while a stream is being captured into a graph.
 * hdof_profile_read waits for the recorded events, writes up to max_out
 * entries (one per kernel name: launches and summed device milliseconds
 * since the previous read) and returns the number of names (or a negative
 * HDOF_E* code); the record is cleared. */
typedef struct hdof_kernel_time {
    char name[32];
    int32_t launches;
    float total_ms;
} hdof_kernel_time;
int hdof_profile(int32_t on);
int hdof_profile_read(hdof_kernel_time* out, int32_t max_out);

/* FP32 arithmetic probe (not in the paper; the measured peak that the
 * ALU-bound kernels are compared against).  Enqueues one kernel of
 * SMs x blocks_per_sm blocks of 256 threads, each running eight independent
 * fused multiply-add chains for iters x 16 steps; *lane_ops (host) receives
 * the number of FMA lane-instructions it executes (blocks x 256 x iters x
 * 128).  Time it with events on `stream`.  sink: device float [256], never
 * written in practice (it keeps the chains from being optimised away). */
int hdof_probe_fma(int32_t blocks_per_sm, int32_t iters, float* sink, double* lane_ops, void* stream);

/* ------------------------------------------------------------ BVH -- */
/* Builds the ray-tracing acceleration structure that stands in for the
 * paper's hardware ray-tracing acceleration (Abstract): a binary BVH built on
 * the GPU by parallel locally-ordered clustering (Meister and Bittner 2018):
 * 63-bit Morton codes of the triangle centroids, radix sort, then rounds
 * that merge mutual nearest neighbours (smallest union-box surface area
 * within 48 positions) until one cluster remains; the triangles are then
 * stored in depth-first leaf order and subtrees of at most two triangles
 * become leaves.
 * verts: float [n_verts][3]; idx: int32 [n_tris][3];
 * mat: float [n_tris][8] = (albedo_a rgb, checker_n, albedo_b rgb, k_s):
 * Lambert diffuse of the albedo, plus for k_s > 0 a white Blinn-Phong
 * highlight k_s sum_l E_l max(0, n . h_l)^32 (h_l the unit half vector of
 * the light and the viewer; lights with n . w_l <= 0 give none);
 * uv: float [n_tris][6] (may be NULL when no material uses a checker).
 * All device pointers; they are read during the call only.  Synchronous
 * with respect to the host (returns once the structure is built).
 * Errors: HDOF_EINVAL (n_tris < 1, bad index), HDOF_ENOMEM, HDOF_ECUDA,
 * HDOF_EUNSUPPORTED (tree deeper than the traversal stack). */
int hdof_build_bvh(const float* verts, int32_t n_verts, const int32_t* idx, int32_t n_tris,
                   const float* mat, const float* uv, hdof_bvh** out, void* stream);
int hdof_bvh_destroy(hdof_bvh* bvh);
int hdof_bvh_info(const hdof_bvh* bvh, hdof_bvh_stats* info);

/* Closest hit of n arbitrary rays (org, dir: float [n][3], dir need not be
 * normalised).  ids: int32 [n] original triangle id or -1; ts: float [n]
 * ray parameter of the hit (unspecified on a miss).  Closest = smallest t;
 * equal t -> lower triangle id (watertight test, edges inclusive, t > 0). */
int hdof_closest_hits(const hdof_bvh* bvh, int32_t n, const float* org, const float* dir,
                      int32_t* ids, float* ts, void* stream);

/* ------------------------------------------------------- G-buffer -- */
/* Deferred-shading G-buffer and sharp image (Design section), rendered as
 * the closest hit of the pinhole ray through each pixel's screen point.
 * Lambert shading: L = albedo (k_a + sum_l E_l max(0, n . w_l)).  prev is
 * the previous frame's camera (pass cam itself for the first frame).
 * hint_tri (device, may be NULL): int32 [H][W] triangle ids likely hit by
 * each pixel's primary ray, e.g. the previous frame's tri plane; it may be
 * out->tri itself (each pixel's hint is read before its id is written).
 * Each primary ray tests its hint first, which only tightens the traversal:
 * any value, including garbage, gives the same G-buffer. */
int hdof_gbuffer(const hdof_bvh* bvh, const hdof_camera* cam, const hdof_camera* prev,
                 const hdof_params* p, const int32_t* hint_tri, const hdof_gbuf* out, void* stream);

/* ---------------------------------------------------- scratch memory -- */
/* Bytes of caller-owned device scratch the calls below need for a
 * width x height frame (one buffer serves them all when they run in order
 * on one stream).  The trace's share grows with
 * p->spp_max: 13 bytes per possible ray (pixel, sample index, record).  The
 * post-filter's region is disjoint from the mask's and the trace's, so
 * hdof_postfilter may run on another stream concurrently with hdof_mask and
 * hdof_trace once hdof_gbuffer has finished. */
size_t hdof_workspace_bytes(int32_t width, int32_t height, const hdof_params* p);

/* ----------------------------------------------------------- mask -- */
/* Adaptive ray mask (Ray Trace section): 5x5 Gaussian (sigma) on the
 * G-buffer normal and depth, 3x3 Sobel scaled by 1/8, edge metric
 * e = max(|grad n|, |grad z| / z~), edge = e > edge_tau; tiles containing an
 * edge, dilated by `dilate` tiles, get spp_max rays per pixel; with
 * variance_on, other pixels whose previous-frame history (nearest pixel at
 * the motion-reprojected position, prev_hist may be NULL) is young or whose
 * luminance std-dev exceeds var_tau get clamp(ceil(spp_max sigma /
 * var_scale), 1, spp_max) rays (spp_max while young).
 * edge, spp: uint8 [H][W] outputs. */
int hdof_mask(const hdof_gbuf* in, const hdof_history* prev_hist, const hdof_params* p,
              uint8_t* edge, uint8_t* spp, void* workspace, size_t workspace_bytes, void* stream);

/* hdof_mask with the ray mask's reach scaled by the CoC (the Discussion's
 * mask resolution scaled by the maximum CoC, against tiling artifacts).
 * With p->mask_coc = 1, each mask tile holding an edge covers the tiles
 * within max(dilate, ceil(r / tile)) tiles of it (Chebyshev distance, at
 * most 8), r = the largest min(|c(z)| / 2, r_max) over the tile's pixels
 * (G-buffer depth, the lens's CoC): every pixel within the blur radius of an
 * edge tile is traced.  With p->mask_coc = 0 it computes what hdof_mask does.
 * cam gives the CoC's image height and tan(fovy/2).  The workspace holds the
 * tile flags and one float per tile (hdof_workspace_bytes covers both).
 * hdof_mask and hdof_mask_noalloc reject mask_coc = 1 (they take no lens). */
int hdof_mask_coc(const hdof_gbuf* in, const hdof_history* prev_hist, const hdof_camera* cam, const hdof_lens* lens,
                  const hdof_params* p, uint8_t* edge, uint8_t* spp, void* workspace, size_t workspace_bytes,
                  void* stream);

/* hdof_mask without caller scratch memory.  The paper has no counterpart:
 * this entry point exists for callers that cannot allocate device memory
 * for the library -- for instance a real-time render thread that must not
 * call cudaMalloc/cudaFree (they can synchronise the device and stall the
 * frame), or a host application that owns all device memory in its own
 * arena and offers plug-ins no allocator.  It computes exactly what
 * hdof_mask computes and allocates nothing: the per-tile flags live in a
 * fixed device array of HDOF_MASK_NOALLOC_MAX_TILES bytes inside the
 * library, which every GPU that loads the library keeps until the process
 * exits.  Frames needing more tiles than that ((W/tile) x (H/tile) rounded
 * up, e.g. 4096x4096 at tile 16) are rejected with HDOF_EINVAL.  The first
 * call on each device looks up the array's device address
 * (cudaGetSymbolAddress) with that device current; make that first call
 * before capturing the stream into a graph.  All calls share the array:
 * calls that overlap on the GPU (different streams without ordering) race
 * and give wrong masks.  Each call clears the tiles it uses first. */
#define HDOF_MASK_NOALLOC_MAX_TILES 65536
int hdof_mask_noalloc(const hdof_gbuf* in, const hdof_history* prev_hist, const hdof_params* p,
                      uint8_t* edge, uint8_t* spp, void* stream);

/* ---------------------------------------------------------- trace */
/* Form and launch shape of the persistent trace (results do not depend on
 * them; hdof_trace takes one optionally, a batch one chosen by an autotuner).
 * trace_block: threads per block (64, 128 or 256);
 * trace_refill: 0 = warp packets (a warp takes 32 consecutive rays of the
 *   list and finds their closest hits in one shared traversal, each lane
 *   culling with its own hit: fast when the rays of neighbouring pixels stay
 *   close, i.e. for small lens apertures); 1..32 = ray level (one ray per
 *   lane; a warp fetches new rays for its idle lanes once fewer than this
 *   many of its 32 lanes still trace); -1 = each view in its default form:
 *   warp packets when the view's CoC scale K = A H / (zf tan(fovy/2)) is
 *   below 20 pixels, ray level with refill 4 otherwise (a batch traces the
 *   two groups of views in two persistent launches, both of trace_block
 *   threads).
 * trace_chunk, spatial_tile: launch granularity of the trace's work queue and
 *   of the batched spatial gather (see the fields).  No choice changes a
 *   result: each ray's closest hit and each pixel's gather are computed the
 *   same way whatever warp or block runs them. */
typedef struct hdof_tuning {
    int32_t trace_block;
    int32_t trace_refill;
    int32_t trace_chunk;   /* queue chunk, 0..16: with packets, packets a warp claims per atomic (0 = 1);
                              ray level, rays per claim in units of 32 (0 = exactly the idle lanes) */
    int32_t spatial_tile;  /* batched spatial reconstruction's pixel tile: 0 or 8 (8x8), or 16 (16x16) */
} hdof_tuning;

/* Thin-lens distributed ray trace of the masked pixels (Ray Trace section).
 * Compacts the pixels with spp > 0 into a queue (tile order) and lists
 * their rays; a persistent kernel traces the ray list (as warp packets or
 * ray by ray, see hdof_tuning), then each queued pixel sums its samples'
 * records in sample order.  min(spp[p], p->spp_max) lens rays
 * per pixel (the ray lists are sized for spp_max): Philox4x32-10
 * (key = (seed, view*65536+frame), counter = (pixel, sample, 0, 0)) gives
 * u1, u2 -> lens point rho = A sqrt(u1), theta = 2 pi u2 (with blades = N:
 * sector k = floor(N u2), f = N u2 - k, point sqrt(u1) ((1-f) V_k + f V_k+1)
 * of the N-gon inscribed in the disk, vertex V_k at angle blade_rot +
 * 2 pi k / N); the ray aims at the pixel's focus-plane point; closest hit;
 * Lambert radiance; split weight w = clamp((c(z) + sqrt2) / (2 sqrt2), 0, 1)
 * into the near layer; each sample weighs 1 + aberration (2 rho^2/A^2 - 1)
 * in every layer sum (hit ratio = weighted near share).
 * rt: float [H][W][12] = (C_near rgb, h | C_far rgb, c_near | P_far xyz,
 * c_far); h = sum w / n is the hit ratio; an empty layer (weight < 1e-6)
 * has colour 0 and CoC -1.  Untraced pixels are not written.
 * hint_tri (device, may be NULL): int32 [H][W] original id of each pixel's
 * primary hit (the G-buffer's tri plane, < 0 for none); each lens ray tests
 * that triangle first, which only tightens the traversal (results do not
 * depend on it).
 * stats (device, may be NULL): uint32 [2] = (traced pixels, rays).
 * rec, ray_off (device, both NULL or both set): per-ray hit records
 * rec[ray_off[p] + s] = (L rgb, view depth of the hit, +inf for a miss) of
 * sample s of traced pixel p -- the frozen visibility that
 * hdof_post_forward/backward re-evaluate at another focus and aperture;
 * rec holds stats[1] float4 entries (at most spp_max x W x H).
 * tune (host, may be NULL): the trace's form and block size (out-of-range
 * values are rejected with HDOF_EINVAL); NULL takes 128 threads and the
 * default form (trace_refill -1): warp packets when the lens's CoC scale
 * K = A H / (zf tan(fovy/2)) is below 20 pixels (|c(z)| = K |zf/z - 1|: the
 * lens rays of neighbouring pixels stay close), ray level with refill 4
 * otherwise. */
int hdof_trace(const hdof_bvh* bvh, const hdof_camera* cam, const hdof_lens* lens,
               const hdof_params* p, const uint8_t* spp, const int32_t* hint_tri, float* rt,
               uint32_t* stats, float* rec, uint32_t* ray_off, void* workspace,
               size_t workspace_bytes, const hdof_tuning* tune, void* stream);

/* Per-ray closest hits of the thin-lens samples (Ray Trace section: each
 * lens ray's closest hit), for checking visibility ray by ray.  Reads the
 * hit records that the last hdof_trace call with this workspace, camera,
 * params and spp left in the workspace (run it on the same stream, before
 * anything else reuses the workspace).  ids: int32 written at
 * [ray_off[p] + s] for sample s of each traced pixel p, where ray_off is the
 * plane that hdof_trace wrote (pass rec/ray_off to it): the original
 * triangle id, or -1 for a miss.  ts (may be NULL): float at the same index,
 * the ray parameter of the hit along the unit direction (+inf for a miss).
 * Both hold at least stats[1] (rays of that trace) entries. */
int hdof_trace_hits(const hdof_bvh* bvh, const hdof_camera* cam, const hdof_params* p, const uint8_t* spp,
                    const void* workspace, size_t workspace_bytes, int32_t* ids, float* ts, void* stream);

/* Full ray-traced depth of field: the quality reference that the paper's
 * Fig. 1 sets beside the hybrid frame (distributed ray tracing of every
 * pixel, no mask, no post-process).  Every pixel is traced with spp_max lens
 * samples per pass (the sampling of hdof_trace); pass k draws its samples
 * with the Philox key of frame (p->frame + k) mod 65536.  out: float
 * [H][W][4] = (mean over the passes of each pass's weighted mean radiance
 * rgb, 0); on the uniform disk (aberration 0) the plain mean of all
 * passes x spp_max samples.
 * workspace: hdof_workspace_bytes(width, height, p) bytes (the post-filter
 * region holds each pass's trace output).  hint_tri as for hdof_trace. */
int hdof_reference_rt(const hdof_bvh* bvh, const hdof_camera* cam, const hdof_lens* lens, const hdof_params* p,
                      int32_t passes, const int32_t* hint_tri, float* out, void* workspace,
                      size_t workspace_bytes, void* stream);

/* Error map between two images a, b (float [H][W][4], rgb compared): err
 * (may be NULL) float [H][W] = mean over rgb of |a - b|; stats: device
 * double [HDOF_ERR_SCRATCH], whose first HDOF_ERR_STATS entries receive
 * (pixels, sum |d|, sum d^2, max |d|) over all pixels, then the same over
 * the pixels where region (uint8 [H][W], may be NULL) is non-zero; sums run
 * over the three channels.  The rest is scratch.  Reduced in a fixed order:
 * the same inputs give the same bits. */
#define HDOF_ERR_STATS 8
#define HDOF_ERR_SCRATCH (HDOF_ERR_STATS + 8 * 1024)
int hdof_error_map(const float* a, const float* b, const uint8_t* region, int32_t width, int32_t height,
                   float* err, double* stats, void* stream);

/* ----------------------------------------------------- post-filter -- */
/* CoC gather post-filter of the sharp image (Design section; the rejection
 * rule of the Reconstruction section).  Scatter-as-gather over soft disks
 * s(r_q - d), s(x) = clamp(x + 1/2, 0, 1), r_q = min(|c(z_q)|/2, r_max),
 * normalised by the disk's lattice area; near layer weighted by w_near(q),
 * far layer by 1 - w_near(q) and the depth test clamp(1 - (z_q - z_p) /
 * (kz_rel z_p), 0, 1).  pp: float [H][W][4] = (alpha N + (1-alpha) F, alpha).
 * Gathers are bounded per 16x16 tile by the largest reaching CoC; where every
 * near source close to a tile has a large CoC, the taps of weight exactly 1
 * are summed from row prefix sums (the same sum, another rounding order).
 * Shaped bokeh (p->blades >= 3 or p->aberration != 0; the Discussion's
 * alternative bokeh shapes and sample weights): the thin lens maps aperture
 * point O of a source at CoC c to the screen offset (c / 2A)(-O_right, O_up),
 * so the soft disk becomes the aperture shape at radius r_q, mirrored
 * left-right for the near layer and top-bottom for the far layer: a source
 * at (dx, dy) from the receiver weighs s(r_q - D(dx, -dy)) (near) or
 * s(r_q - D(-dx, dy)) (far) times 1 + aberration (2 min(d / r_q, 1)^2 - 1)
 * (1 while r_q < 1), D the aperture norm (hdof_params.blades), normalised by
 * that shape's lattice area; computed by a separate gather (no row-prefix
 * interior).  Not available in batches or the differentiable path. */
int hdof_postfilter(const hdof_gbuf* in, const hdof_camera* cam, const hdof_lens* lens,
                    const hdof_params* p, float* pp, void* workspace, size_t workspace_bytes,
                    void* stream);

/* ------------------------------------------------- reconstruct -- */
/* Spatio-temporal reconstruction (Reconstruction section).  Temporal: near
 * terms and moments reprojected by mv, far terms by the previous-frame
 * projection of the far position (own far hits, else the 3x3 neighbours',
 * else the G-buffer point); bilinear over taps with history, invalid below
 * weight 1e-3; EMA with ema_alpha, or with alpha_k > 0 a per-pixel weight
 * (the Discussion's per-pixel blend factors against ghosting): lambda = the
 * larger of clamp((|Y - mu1| - alpha_k sigma_L) / max(Y, mu1, 1e-3), 0, 1)
 * (this frame's ray-traced luminance Y against the reprojected history
 * moments) and clamp(|h - B_near| - alpha_k sqrt(B_near (1 - B_near) / spp),
 * 0, 1) (the hit ratio against its reprojected EMA), alpha = ema_alpha +
 * (1 - ema_alpha) lambda; layer colours normalised by their
 * accumulated hit ratio; composed with this frame's hit ratio when
 * camera_moved, else the accumulated one; CoC = H_acc c_near + (1-H_acc)
 * c_far.  Spatial: for traced pixels, gather of traced neighbours with
 * weight s(r_p - d) s(r_q - d), r = min(c/2, r_s), blended by
 * beta = clamp(sigma_L / var_ref, 0, 1) (1 while hlen < 2).
 * hist_in (previous frame) is read, hist_out written; they must differ.
 * crt: float [H][W][4] (C_rt rgb, c_rt), untraced pixels (0,0,0,-1);
 * hacc: float [H][W] accumulated hit ratio; crec: float [H][W][4]
 * (C_rec rgb, 0).  hacc and crec are written for traced pixels only. */
int hdof_reconstruct(const float* rt, const hdof_gbuf* in, const uint8_t* spp,
                     const hdof_camera* cam, const hdof_camera* prev, const hdof_lens* lens,
                     const hdof_params* p, const hdof_history* hist_in,
                     const hdof_history* hist_out, float* crt, float* hacc, float* crec,
                     void* stream);

/* ------------------------------------------------------- composite -- */
/* Composite (Composite section): focus weight f = clamp(sqrt2 + 1/2 - c, 0,
 * 1) with c the reconstructed CoC where traced, else |c(z)|; near branch
 * = C_rec where traced, else C_pp; far branch = lerp(C_rec, C_pp,
 * clamp(H_acc / h_tau, 0, 1)) where traced, else C_pp; blended by
 * w_near(c(z)); out = lerp(blur, sharp, f).  out: float [H][W][4]. */
int hdof_composite(const hdof_gbuf* in, const uint8_t* spp, const float* pp, const float* crt,
                   const float* crec, const float* hacc, const hdof_camera* cam,
                   const hdof_lens* lens, const hdof_params* p, float* out, void* stream);

/* Specular-bokeh preference (Composite section): bright specular bokeh is
 * taken from the post-process rather than the noisy ray trace, by the
 * intensity of the post-process colour's specular part.
 * hdof_postfilter_spec: that specular part, the post-filter of
 * hdof_postfilter applied to the plane (S, S, S) of the G-buffer's col.w in
 * place of the colour (the filter is linear in the colour, so this is
 * exactly the share of S in pp).  pp_spec: float [H][W][4] = (S_pp, S_pp,
 * S_pp, alpha).  workspace as for hdof_postfilter, whose first 16 bytes per
 * pixel (the mask's and the trace's region) hold the grey plane: unlike
 * hdof_postfilter it must not run concurrently with hdof_mask, hdof_trace or
 * hdof_postfilter on the same workspace.
 * hdof_composite_spec: hdof_composite whose near branch where traced is
 * lerp(C_rec, C_pp, clamp(spec_pref S_pp, 0, 1)); pp_spec may be NULL and
 * is ignored when spec_pref = 0 (then it equals hdof_composite).  Neither
 * is batched; the differentiable path rejects spec_pref != 0
 * (HDOF_EUNSUPPORTED). */
int hdof_postfilter_spec(const hdof_gbuf* in, const hdof_camera* cam, const hdof_lens* lens,
                         const hdof_params* p, float* pp_spec, void* workspace, size_t workspace_bytes,
                         void* stream);
int hdof_composite_spec(const hdof_gbuf* in, const uint8_t* spp, const float* pp, const float* pp_spec,
                        const float* crt, const float* crec, const float* hacc, const hdof_camera* cam,
                        const hdof_lens* lens, const hdof_params* p, float* out, void* stream);

/* ------------------------------------------------- batched multi-view -- */
/* One view of a batch: its scene, cameras, lens, constants and buffers
 * (every pointer as for the single-view calls; FP32 G-buffer planes, mv
 * required).  hist_in is the previous frame's history (hlen = 0 everywhere
 * for none), hist_out the one this frame writes.  workspace: at least
 * hdof_workspace_bytes(width, height, &params) bytes, one per view.
 * stats may be NULL. */
typedef struct hdof_view {
    const hdof_bvh* bvh;
    hdof_camera cam, prev;
    hdof_lens lens;
    hdof_params params;
    hdof_gbuf g;
    uint8_t* edge;
    uint8_t* spp;
    float* rt;
    uint32_t* stats;
    float* pp;
    float* crt;
    float* hacc;
    float* crec;
    float* out;
    hdof_history hist_in, hist_out;
    void* workspace;
    size_t workspace_bytes;
} hdof_view;


typedef struct hdof_batch hdof_batch;

/* Prepares a batch: validates every view, builds each stage's per-view
 * launch records and block tables and copies them to device memory the
 * handle owns (synchronous).  The views' buffers must stay valid while the
 * handle is used.  tuning may be NULL (128 threads,
 * each view's trace in its default form: trace_refill -1).  Views with
 * shaped bokeh or spec_pref != 0 return HDOF_EUNSUPPORTED (specular
 * materials themselves are shaded as in the single-view calls). */
int hdof_batch_create(const hdof_view* views, int32_t n_views, const hdof_tuning* tuning, hdof_batch** out,
                      void* stream);
int hdof_batch_destroy(hdof_batch* batch);
/* Rewrites the launch records for the next frame (cameras, lens, params,
 * history ping-pong, even the BVH) from views[0..n_views), which must keep
 * the count, sizes and mask tile the batch was created with.  The records
 * are uploaded from a pinned host image with one asynchronous copy on
 * stream, so a CUDA graph captured from hdof_batch_render stays valid and
 * replays the new frame when launched after this call on the same stream.
 * Renders enqueued on another stream must be ordered by the caller. */
int hdof_batch_update(hdof_batch* batch, const hdof_view* views, int32_t n_views, void* stream);
/* Bytes of the launch records each hdof_batch_update uploads (0 for NULL). */
size_t hdof_batch_bytes(const hdof_batch* batch);
/* Enqueues the frame of every view of the batch: one launch per stage over
 * all views' blocks (G-buffer, mask, compaction, one persistent trace over
 * the concatenated ray queues -- two, one per form, when each view takes
 * its default form (trace_refill -1) -- post-filter, reconstruction,
 * composite).
 * The frame is forked from `stream` onto two streams the handle owns: the
 * critical path (highest priority) and the post-filter (lowest), forked
 * after the G-buffer and joined before the composite, so the post-filter
 * runs concurrently with the mask, compaction, trace and reconstruction;
 * the frame is joined back to `stream` at its end.  Only kernel launches,
 * device memsets and event forks and joins: capturable into a CUDA graph.  Each view's results equal
 * those of the single-view calls bit for bit. */
int hdof_batch_render(const hdof_batch* batch, void* stream);

/* The batched frame's stages, in order; hdof_batch_render runs all of them. */
enum {
    HDOF_STAGE_GBUFFER = 0,     /* 1 launch */
    HDOF_STAGE_MASK = 1,        /* tile clear, edge, spp: 3 launches */
    HDOF_STAGE_COMPACT = 2,     /* count, scan, scatter: 3 launches */
    HDOF_STAGE_TRACE = 3,       /* ray prefix, persistent trace, resolve: 3 launches (5 with per-view forms) */
    HDOF_STAGE_POSTFILTER = 4,  /* prep, row prefix, gather: 3 launches */
    HDOF_STAGE_RECONSTRUCT = 5, /* temporal, spatial: 2 launches */
    HDOF_STAGE_COMPOSITE = 6,   /* 1 launch */
    HDOF_BATCH_STAGES = 7
};
/* Enqueues stages first..last (inclusive) of the batched frame, e.g. to time
 * them one by one or to interleave the caller's own work; running 0..6 in
 * order, in one call or several, is hdof_batch_render. */
int hdof_batch_render_range(const hdof_batch* batch, int32_t first, int32_t last, void* stream);

/* ------------------------------------------- differentiable post-path -- */
/* Buffers the forward writes and the backward reads (device, FP32 unless
 * noted; [H][W] planes): rt [12] trace output replayed at this lens; crt [4],
 * hacc, mom [2], hlen (uint8) of the temporal step; crec [4] and sp_aux [4]
 * (gathered colour, weight sum) of the spatial gather; pp [4] and pp_aux
 * [8] (near colour, near weight, far colour, far weight) of the post-filter;
 * out [4] the composite. */
typedef struct hdof_post_state {
    float* rt;
    float* crt;
    float* hacc;
    float* mom;
    uint8_t* hlen;
    float* crec;
    float* sp_aux;
    float* pp;
    float* pp_aux;
    float* out;
} hdof_post_state;

/* Scratch bytes of hdof_post_forward / hdof_post_backward. */
size_t hdof_post_workspace_bytes(int32_t width, int32_t height, const hdof_params* p);

/* The frame's reconstruction, post-filter and composite as a function of the
 * sharp colour image (in->col, FP32) and of the lens, with the ray-traced
 * visibility held fixed (the paper has no gradient; this exposes one).
 * Frozen inputs: in->nd (view depth in .w), spp, the hit records rec /
 * ray_off of an hdof_trace call with the same spp, and hist_samples
 * ([H][W][12]: near (rgb x B, B), far (rgb x B, B), mu1, mu2,
 * valid_near + 2 valid_far, hlen -- the history already sampled at its
 * reprojected positions; NULL = no history).  The trace accumulation is
 * re-evaluated from the records at `lens` (each hit's CoC and split weight
 * change, not the hits), then the temporal step over the frozen samples, the
 * spatial gather, the post-filter and the composite run with the frame's
 * definitions.  Writes every buffer of *st: rt, hacc, mom, crec and sp_aux
 * at the traced pixels only, the others at every pixel. */
int hdof_post_forward(const hdof_gbuf* in, const uint8_t* spp, const float* rec, const uint32_t* ray_off,
                      const float* hist_samples, const hdof_camera* cam, const hdof_lens* lens,
                      const hdof_params* p, const hdof_post_state* st, void* workspace,
                      size_t workspace_bytes, void* stream);

/* Adjoint of hdof_post_forward (same inputs, its state): from grad_out
 * ([H][W][4], rgb used) writes grad_col ([H][W][4], d/d colour) and
 * grad_lens (device float [2] = d/d focus_dist, d/d aperture_radius).  Gather
 * weights are recomputed, not stored; the lens gradient is reduced per block
 * in double precision and summed in a fixed order (deterministic).  Needs
 * aperture_radius > 0.  Both calls take the fixed EMA weight, the uniform
 * circular lens and no specular preference: alpha_k, blades, aberration and
 * spec_pref other than 0 return HDOF_EUNSUPPORTED. */
int hdof_post_backward(const hdof_gbuf* in, const uint8_t* spp, const float* rec, const uint32_t* ray_off,
                       const float* hist_samples, const hdof_camera* cam, const hdof_lens* lens,
                       const hdof_params* p, const hdof_post_state* st, const float* grad_out,
                       float* grad_col, float* grad_lens, void* workspace, size_t workspace_bytes,
                       void* stream);

/* hdof_post_forward / hdof_post_backward with the lens on the device:
 * lens_dev = device float [2] (focus distance, aperture radius), read by the
 * kernels when they run, so that a fitting step needs no read-back of the
 * lens to the host and can be captured into a CUDA graph (each replay reads
 * the array's values then).  Results are those of the host-record calls
 * with the same lens, bit for bit (the CoC constants are computed with the
 * same single-precision arithmetic).  The values are not checked on the
 * host: a focus distance or aperture that is not finite and positive gives
 * non-finite outputs (every access stays in bounds).  lens_dev NULL:
 * HDOF_EINVAL; every other argument as in the host-record calls. */
int hdof_post_forward_dlens(const hdof_gbuf* in, const uint8_t* spp, const float* rec, const uint32_t* ray_off,
                            const float* hist_samples, const hdof_camera* cam, const float* lens_dev,
                            const hdof_params* p, const hdof_post_state* st, void* workspace,
                            size_t workspace_bytes, void* stream);
int hdof_post_backward_dlens(const hdof_gbuf* in, const uint8_t* spp, const float* rec, const uint32_t* ray_off,
                             const float* hist_samples, const hdof_camera* cam, const float* lens_dev,
                             const hdof_params* p, const hdof_post_state* st, const float* grad_out,
                             float* grad_col, float* grad_lens, void* workspace, size_t workspace_bytes,
                             void* stream);

#ifdef __cplusplus
}
#endif
#endif /* HDOF_H */
