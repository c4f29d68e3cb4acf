/*
 * vtx.h -- C ABI of the GB300 meshless molecular ray-caster.
 *
 * The paper (VTX, Methods: "Meshless Representations", "High Quality
 * Rendering") draws a molecule -- atom positions, radii and connectivity --
 * without triangle meshes: every primitive (a van der Waals sphere, or the
 * spheres and bond cylinders of ball-and-stick) is ray-cast against its
 * implicit surface so that each pixel shows the nearest hit, and lighting is
 * deferred: shading and screen-space ambient occlusion run on the per-pixel
 * hit record.  This library computes that per-frame path on one GPU with
 * hand-written CUDA kernels for sm_103a:
 *
 *   cull -> precise setup / direct splat -> tile binning + per-tile depth
 *   sort -> tile ray-cast -> resolve (depth, id, normal) -> Blinn-Phong
 *   shading -> SSAO,
 *
 * plus a batched form for molecular-dynamics trajectories (many frames x
 * views per call, optionally replayed as one CUDA graph) and a soft-edge
 * differentiable form with a hand-written backward pass.
 *
 * Conventions (shared by every entry point):
 *   - Atoms are float4 records (x, y, z, r) in Angstrom, world space.
 *   - Camera: float32 eye and basis used exactly as passed (not
 *     re-normalised).  Pixel (px, py), row 0 at the TOP, has its ray through
 *     the pixel centre: slope a = (px + 0.5 - W/2)/f, b = (H/2 - py - 0.5)/f
 *     with f = H / (2 tan_half_fovy).  Depth is the distance along the
 *     forward axis; a hit is accepted only when its entry point lies at or
 *     beyond znear (an entry point in front of znear skips the primitive).
 *   - Normals are reported in the right-handed view frame (x right, y up,
 *     z toward the viewer).
 *   - Output planes are caller-owned buffers laid out [H][W] (normal and
 *     rgb: [3][H][W], one plane per component), in device memory or, for
 *     vtx_render_frame, page-locked host memory (written over the host
 *     link by the resolve kernel).
 *   - Background pixels: depth +inf, id 0xFFFFFFFF, normal 0, rgb =
 *     settings.background, ao 1.
 *   - Primitive ids: atoms 0..n_atoms-1; bond b (ball-and-stick) is
 *     n_atoms + b.  Equal depths resolve to the smaller id.
 *
 * Ownership and asynchrony: pointers given to vtx_upload_* are
 * recorded, not copied; the caller keeps them alive and unchanged until the
 * next upload or vtx_destroy.  Every render call only enqueues work on the
 * context's stream and returns; results are ready after the caller
 * synchronises that stream.  The context owns and grows its scratch memory.
 *
 * Errors: every call returns a vtx_status; vtx_last_error() gives the text
 * of the most recent failure.  Argument errors are detected on the host
 * before anything is enqueued.  Capacity overflows of the scratch arena are
 * detected on the device (the kernels stop writing past a capacity and
 * record the size they needed); the next vtx_sync_status() (or a render
 * call with VTX_FLAG_SYNC) reports VTX_ERR_CAPACITY once and grows the arena
 * so that re-rendering succeeds.  No kernel waits on another block or launch;
 * the only device-side waits are bounded polls on the completion of the
 * kernel's own bulk copies (VTX_ERR_TIMEOUT if one ever gives up).
 */
#ifndef VTX_H_
#define VTX_H_

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct vtx_ctx vtx_ctx;

typedef enum {
  VTX_OK = 0,
  VTX_ERR_INVALID_ARG = 1, /* a null pointer, a size out of range, an unsupported mode */
  VTX_ERR_CUDA = 2,        /* a CUDA runtime call failed (text in vtx_last_error) */
  VTX_ERR_OOM = 3,         /* device allocation of scratch memory failed */
  VTX_ERR_CAPACITY = 4,    /* a previous frame overflowed the scratch arena (now grown: render again) */
  VTX_ERR_TIMEOUT = 5,     /* a bounded device-side wait for a bulk copy gave up; the frame is invalid */
  VTX_ERR_BOUNDS = 6,      /* a device-side bounds check failed: a decoded primitive id out of range */
  VTX_ERR_STATE = 7        /* call order: no atoms uploaded, no camera set */
} vtx_status;

/* Representations (the paper's meshless list, Methods "Meshless Representations"). */
enum {
  VTX_MODE_VDW = 0,             /* van der Waals: spheres of radius xyzr.w */
  VTX_MODE_BALL_AND_STICK = 1,  /* spheres of radius ball_radius + bond cylinders of radius bond_radius */
  VTX_MODE_STICKS = 2,          /* spheres and bond cylinders, all of radius bond_radius */
  VTX_MODE_SAS = 3              /* solvent accessible surface: spheres of radius xyzr.w + probe_radius */
};

/* Shading models (the paper's list, "High Quality Rendering": flat, matte, glossy, toon). */
enum {
  VTX_SHADE_GLOSSY = 0,  /* Blinn-Phong: albedo (ka + kd max(n.L,0)) + ks [n.L>0] max(n.H,0)^shininess */
  VTX_SHADE_FLAT = 1,    /* albedo */
  VTX_SHADE_MATTE = 2,   /* albedo (ka + kd max(n.L,0)) */
  VTX_SHADE_TOON = 3     /* albedo (ka + kd b), b = min(floor(max(n.L,0) L), L-1) / (L-1), L = toon_levels */
};

enum {
  VTX_FLAG_SYNC = 1u,     /* synchronise at the end of the call and report device-side errors */
  VTX_FLAG_PROFILE = 2u,  /* record per-stage CUDA events (read with vtx_stage_times) */
  VTX_FLAG_NO_SSAO = 4u,  /* skip ambient occlusion even if ssao_samples > 0 */
  VTX_FLAG_PROFILE_CULL = 8u, /* record CUDA events around the cull stage only (vtx_stage_times reports its
                                time, the other stages 0): two events per frame instead of nine, so the
                                other kernels keep their overlapped launches */
  VTX_FLAG_SOFT_REUSE = 16u   /* soft backward only: the caller vouches that the contents of xyzr are those
                                of the latest soft forward call on this context (see vtx_render_soft_bwd_ex) */
};

/* Pinhole camera, 64 bytes.  forward/right/up: the view basis (float32 as passed). */
typedef struct {
  float eye[3];
  float forward[3];
  float right[3];
  float up[3];
  float tan_half_fovy; /* tan of half the VERTICAL field of view */
  float znear;         /* near plane depth, > 0 */
  int32_t width;       /* pixels, 1..16384 */
  int32_t height;      /* pixels, 1..16384 */
} vtx_camera;

#define VTX_MAX_SSAO_SAMPLES 64
#define VTX_MAX_ELEMENTS 32
#define VTX_MAX_VIEWS 16

/*
 * Rendering settings.  vtx_default_settings() fills the values used by the
 * tests: glossy (Blinn-Phong) ka 0.2, kd 0.7, ks 0.3, shininess 32, light
 * (0.25, 0.5, 1) in view space, white background, no SSAO, 16x16 tiles,
 * direct splat up to 16 candidate pixels (tile_w = 0 lets the library
 * autotune both), 4 toon bands, SAS probe 1.4 A, no clipping, fog or outline.
 * The paper names these techniques but not their constants.  Order of the
 * per-pixel operations: shade, times AO, outline (replaces the colour), fog.
 */
typedef struct {
  int32_t mode;          /* VTX_MODE_* */
  float ball_radius;     /* ball-and-stick sphere radius (A) */
  float bond_radius;     /* ball-and-stick cylinder radius (A) */
  float ka, kd, ks, shininess;
  float light_dir[3];    /* view space; normalised by the library */
  float background[3];
  int32_t ssao_samples;  /* 0 = off, else 1..VTX_MAX_SSAO_SAMPLES */
  float ssao_radius;     /* A */
  float ssao_bias;       /* A */
  float ssao_kernel[VTX_MAX_SSAO_SAMPLES][3]; /* hemisphere offsets (unit-ball scale), z along the normal */
  int32_t tile_w, tile_h; /* 16x16, 32x8 or 8x8; tile_w = 0: autotune tile shape AND splat_max_px (below) */
  int32_t splat_max_px;  /* primitives whose candidate pixel box is <= this are splatted directly; 0 = the
                            library default: 4 when the primitives number at most one per 8 pixels, else 16
                            (the planes are the same for every value) */
  uint32_t flags;        /* VTX_FLAG_* */
  /* post-processes and variants (the paper's list: shading modes, fog, outline; Fig. 1C clipping) */
  int32_t shading;       /* VTX_SHADE_* */
  int32_t toon_levels;   /* VTX_SHADE_TOON: number of diffuse bands, 2..16 */
  float probe_radius;    /* VTX_MODE_SAS: added to every atom radius (A) */
  float clip_plane[4];   /* (nx, ny, nz, d), world space: atoms with n.x + d < 0 are removed (bonds with
                            either atom removed too); n = 0 disables */
  float fog_near, fog_far; /* linear fog over this depth range (A) toward the background colour */
  float fog_density;     /* fog weight at fog_far and beyond, in [0,1]; 0 disables */
  float outline_depth;   /* A: a covered pixel whose 4-neighbour is background or deeper by more than this
                            takes outline_color; 0 disables */
  float outline_color[3];
} vtx_settings;

/* Output planes (caller-owned; device or, for vtx_render_frame, page-locked host memory).  ao may be NULL. */
typedef struct {
  float *depth;     /* [H][W] depth of the visible hit, +inf for background */
  uint32_t *id;     /* [H][W] primitive id, 0xFFFFFFFF for background */
  float *normal;    /* [3][H][W] unit normal, right-handed view frame */
  float *rgb;       /* [3][H][W] shaded colour times ambient occlusion, in [0,1] */
  float *ao;        /* [H][W] ambient occlusion factor in [0,1] (1 when SSAO is off) */
} vtx_outputs;

/* Version string of the library. */
const char *vtx_version(void);

/* Fill *s with the defaults listed above. */
vtx_status vtx_default_settings(vtx_settings *s);

/*
 * A rendering context: the per-frame engine state of the paper's Molecular
 * Graphics Engine (Methods; Implementation: one engine drawing the molecule
 * every frame) -- the recorded molecule, the camera and the scratch memory
 * the frame pipeline reuses from frame to frame.
 *
 * vtx_create: a context on CUDA device `device` (0..device count - 1, else
 * VTX_ERR_INVALID_ARG; *out is set to NULL on failure).  `cuda_stream` is a
 * cudaStream_t owned by the caller (NULL = the legacy default stream).
 * Allocates only a few small host-pinned and device buffers (VTX_ERR_OOM
 * when that fails); scratch grows on first use.
 * vtx_destroy: synchronises the context's stream, then frees everything the
 * context owns (never the caller's arrays or stream).  VTX_ERR_INVALID_ARG
 * for NULL.
 * vtx_set_stream: later calls enqueue on `cuda_stream`; cached batch graphs
 * are dropped (they were captured on the previous stream).
 */
vtx_status vtx_create(vtx_ctx **out, int32_t device, void *cuda_stream);
vtx_status vtx_destroy(vtx_ctx *ctx);
vtx_status vtx_set_stream(vtx_ctx *ctx, void *cuda_stream);

/*
 * Record the atom set (the molecule of the paper's Methods: positions, radii).
 * xyzr: float4 [n_atoms]; elem: uint8 [n_atoms] element index (< n_elem),
 * may be NULL (element 0); palette_rgb: HOST float [n_elem][3] element
 * colours (copied).  n_atoms in 0..2^31-1, n_elem in 1..32.  Not copied: the
 * arrays must stay valid and unchanged while frames render.
 *
 * xyzr and elem may be device memory or PAGE-LOCKED host memory
 * (cudaHostAlloc / cudaHostRegister).  Host-resident atoms are read by the
 * kernels over the host link every frame (the streaming cull reads each
 * record once; setup and resolve read only survivors and visible atoms), so
 * the atom count is bounded by host memory, not device memory: the
 * out-of-core form of the paper's Performance evaluation (several hundred
 * million atoms, streamed).  Pageable host memory returns
 * VTX_ERR_INVALID_ARG.  The same rule holds for vtx_upload_bonds pairs and
 * vtx_render_batch frames.
 */
vtx_status vtx_upload_atoms(vtx_ctx *ctx, const float *xyzr, const uint8_t *elem, const float *palette_rgb,
                            int32_t n_elem, int64_t n_atoms);

/*
 * Record the connectivity (the paper's "connectivity"; drawn as capped
 * cylinders in ball-and-stick and sticks).  pairs: uint32 [n_bonds][2]
 * (device or page-locked host memory), i < j <
 * n_atoms, endpoints at least 1e-3 A apart.  n_bonds = 0 clears them.
 */
vtx_status vtx_upload_bonds(vtx_ctx *ctx, const uint32_t *pairs, int64_t n_bonds);

/*
 * Set the camera for vtx_render_frame (copied).  The paper's interaction
 * modes (Improved user experience: trackball and free-fly cameras) end in
 * one pinhole camera per frame; this is that camera, with the conventions
 * stated at the top of this header.  VTX_ERR_INVALID_ARG when a size is
 * outside 1..16384, tan_half_fovy or znear is not finite and positive, or a
 * component of the eye or the basis is not finite.
 */
vtx_status vtx_set_camera(vtx_ctx *ctx, const vtx_camera *cam);

/*
 * Render one frame of the recorded atoms from the current camera: the
 * nearest hit per pixel (ids exact), its depth and normal, Blinn-Phong
 * shading and, when settings->ssao_samples > 0, SSAO.  Enqueued on the
 * context's stream.
 */
vtx_status vtx_render_frame(vtx_ctx *ctx, const vtx_settings *s, const vtx_outputs *out);

/*
 * Same as vtx_render_frame, with HOST inputs and outputs: copies xyzr and
 * elem (host, pinned recommended) to context-owned device memory, renders,
 * and copies every output plane back into host buffers (same layout as
 * vtx_outputs).  Synchronises before returning.  Used to measure end to end
 * throughput including host<->device traffic.
 */
vtx_status vtx_render_frame_host(vtx_ctx *ctx, const float *xyzr_host, const uint8_t *elem_host,
                                 const float *palette_rgb, int32_t n_elem, int64_t n_atoms,
                                 const vtx_camera *cam, const vtx_settings *s, const vtx_outputs *out_host);

/*
 * Batched trajectory rendering (the paper: trajectories re-rendered every
 * frame, ambient occlusion included).  frames_xyzr: float4
 * [n_frames][frame_stride] in device or page-locked host memory (a
 * trajectory larger than device memory streams from the host); frame f uses
 * its first atom_counts[f] records;
 * atom_counts: HOST int64 [n_frames], uneven allowed, each <= frame_stride;
 * the element array of vtx_upload_atoms is indexed by atom (must cover
 * frame_stride atoms, or be NULL).  cams: HOST [n_views] cameras, all with
 * the same width and height, n_views <= VTX_MAX_VIEWS.  out: ONE vtx_outputs
 * whose planes hold n_frames*n_views images back to back, image index
 * f*n_views + v (plane stride H*W, normal/rgb 3*H*W per image).
 * VTX_MODE_VDW or VTX_MODE_SAS (no bonds).  use_graph != 0 captures the whole batch into a CUDA
 * graph on first use and replays it on later calls with identical
 * arguments (one cudaGraphLaunch per call).
 */
vtx_status vtx_render_batch(vtx_ctx *ctx, const float *frames_xyzr, int64_t frame_stride,
                            const int64_t *atom_counts, int32_t n_frames, const vtx_camera *cams,
                            int32_t n_views, const vtx_settings *s, const vtx_outputs *out, int32_t use_graph);

/*
 * Soft-edge (differentiable) renderer, forward.  Per pixel, over the spheres
 * whose signed pixel distance to the silhouette is >= -4 px, ordered by
 * centre depth (ties: smaller id), front-to-back composite of
 * alpha = min(0.99, sigmoid(delta_px / sigma_px)), stopping once the
 * transmittance falls below 1e-4.  Outputs per view v: coverage [V][H][W],
 * depth [V][H][W] (sum of w_i t_i), normal [V][3][H][W] (sum of w_i n_i, view
 * frame).  xyzr: device float4 [n]; cams: HOST [n_views], equal sizes.
 */
vtx_status vtx_render_soft_fwd(vtx_ctx *ctx, const float *xyzr, int64_t n, const vtx_camera *cams,
                               int32_t n_views, float sigma_px, float *cov, float *depth, float *normal);

/*
 * Soft-edge renderer, backward: grad_xyzr (device float4 [n], 16-byte aligned, OVERWRITTEN;
 * VTX_ERR_INVALID_ARG when NULL or unaligned, before any launch)
 * = d/d(x,y,z,r) of sum over views and pixels of
 *   g_cov*cov + g_depth*depth + g_normal . normal.
 * Tile lists are rebuilt (vtx_render_soft_bwd_ex can reuse the forward
 * call's lists).  Gradient planes have the layout of the forward outputs;
 * any may be NULL (zero).
 */
vtx_status vtx_render_soft_bwd(vtx_ctx *ctx, const float *xyzr, int64_t n, const vtx_camera *cams,
                               int32_t n_views, float sigma_px, const float *g_cov, const float *g_depth,
                               const float *g_normal, float *grad_xyzr);

/*
 * The two soft-edge calls above with a flags word and an optional per-pixel
 * state.  flags: VTX_FLAG_SYNC makes the call synchronise and, after a
 * capacity overflow, grow the arena and render again (what
 * vtx_render_soft_fwd / _bwd always do).  Without it the first call of a
 * problem size (atoms, views, W, H) on a context still does that, and later
 * calls only enqueue: a device-side error is then reported by the next
 * vtx_sync_status() (or synchronising call), and the outputs of the call
 * that raised it are invalid.
 * state: NULL, or uint32 [n_views][H][W][2], 8-byte aligned, caller-owned.
 * The forward call writes per pixel the final transmittance (float bits)
 * and 1 + the position of its last contributor in the tile's sorted list;
 * a backward call given the state of the forward call made with the SAME
 * xyzr, cams and sigma_px skips its front-to-back walk.  Any other state
 * gives wrong gradients.
 * The forward call leaves its tile lists, in their sorted order, in the
 * context's arena.  A backward call with VTX_FLAG_SOFT_REUSE reuses them
 * (no cull, binning or sort) when that forward call was the context's latest
 * call to use the arena, with the same xyzr pointer, n, cams (compared byte
 * for byte) and sigma_px, and no context buffer has been reallocated since;
 * otherwise it rebuilds them, as without the flag.  The flag is the caller's
 * promise that the CONTENTS of xyzr have not changed since that forward call
 * (the library compares only the pointer); a broken promise gives wrong
 * gradients.  The flag is ignored by forward calls.
 */
vtx_status vtx_render_soft_fwd_ex(vtx_ctx *ctx, const float *xyzr, int64_t n, const vtx_camera *cams,
                                  int32_t n_views, float sigma_px, uint32_t flags, float *cov, float *depth,
                                  float *normal, uint32_t *state);
vtx_status vtx_render_soft_bwd_ex(vtx_ctx *ctx, const float *xyzr, int64_t n, const vtx_camera *cams,
                                  int32_t n_views, float sigma_px, uint32_t flags, const float *g_cov,
                                  const float *g_depth, const float *g_normal, const uint32_t *state,
                                  float *grad_xyzr);

/*
 * Number of sigmoid terms the most recent soft forward call composited,
 * summed over its pixels (the oracle's contributor count: spheres within
 * -4 px of their silhouette, front to back until the transmittance stop).
 * This is the forward pass's algorithmic work, used for its FP32 roofline.
 * Synchronises.
 */
vtx_status vtx_soft_terms(vtx_ctx *ctx, uint64_t *n_terms);

/*
 * Headless image export (Methods, High Quality Rendering: images up to 8K
 * with a custom background of user-defined transparency): packs rendered
 * planes into interleaved 8-bit RGBA.  R, G, B = round-to-nearest-even(255 *
 * clamp(c, 0, 1)) of the rgb planes (shading, AO, outline and fog included);
 * A = 255 where a primitive was hit (id != 0xFFFFFFFF), else
 * round-to-nearest-even(255 * clamp(background_alpha, 0, 1)) (straight
 * alpha: background pixels keep the background colour in R, G, B).  rgb:
 * float [n_images][3][H][W] and id: uint32 [n_images][H][W] as written by
 * vtx_render_frame / vtx_render_batch; rgba: uint8 [n_images][H][W][4],
 * 4-byte aligned.  All three may be device or page-locked host memory (a
 * host rgba buffer is written over the host link, 4 bytes per pixel instead
 * of the planes' 36).  Enqueued on the context's stream; W, H in 1..16384
 * (8K = 7680 x 4320).
 */
vtx_status vtx_export_rgba8(vtx_ctx *ctx, const float *rgb, const uint32_t *id, int32_t width, int32_t height,
                            int32_t n_images, float background_alpha, uint8_t *rgba);

/*
 * Solvent excluded surface (Methods, "Cartoon and SES representations": the
 * SES is computed by a discrete approach and extracted with marching cubes).
 * Grid point (i, j, k) is origin + spacing * (i, j, k).
 */
typedef struct {
  float origin[3];  /* world position of grid point (0, 0, 0), A */
  float spacing;    /* h > 0, A */
  int32_t dims[3];  /* grid points along x, y, z, each >= 2; product <= 2^32 */
  float probe;      /* probe radius p >= 0, A; p / h <= 150 */
} vtx_ses_grid;

/*
 * A grid covering every atom's solvent accessible sphere (radius r + probe)
 * with two spare points on each side: origin = min(c - r - p) - 2 h, dims =
 * floor((max(c + r + p) - min(c - r - p)) / h) + 6.  xyzr: float4 [n_atoms],
 * device or page-locked host memory.  Synchronises.
 */
vtx_status vtx_ses_fit_grid(vtx_ctx *ctx, const float *xyzr, int64_t n_atoms, float probe, float spacing,
                            vtx_ses_grid *grid);

/*
 * The SES of the atoms on `grid` as a triangle soup.  Definitions:
 *   SAS interior: point X is inside when some atom (c, r) has
 *     ((X-c)_x^2 + (X-c)_y^2) + (X-c)_z^2 < (r + p)^2, evaluated in FP64 with
 *     every operation correctly rounded in this order (X = (double)origin +
 *     (double)h * i per axis);
 *   edt2: squared distance in grid units to the nearest grid point outside
 *     the SAS interior, exact when <= K^2 (K = ceil(p / h) + 1), else K^2 + 1;
 *   SES interior: edt2 >= 1 and edt2 * h^2 >= p^2 (FP64; with p = 0 the
 *     SES is the union of the spheres);
 *   marching cubes over the cells, cell order i fastest then j then k; per
 *     cell, loops of crossing edges (a face with four crossings cuts its
 *     inside corners apart), each running counter-clockwise about the
 *     outward normal (inside to outside), starting at its smallest edge
 *     (corners 0 (0,0,0), 1 (1,0,0), 2 (1,1,0), 3 (0,1,0), 4 (0,0,1),
 *     5 (1,0,1), 6 (1,1,1), 7 (0,1,1); edges 0-3 the z = 0 square 0-1, 1-2,
 *     2-3, 3-0, edges 4-7 the z = 1 square 4-5, 5-6, 6-7, 7-4, edges 8-11
 *     the verticals 0-4, 1-5, 2-6, 3-7); a
 *     three-edge loop is one triangle, a longer loop of L edges L triangles
 *     around the mean of its vertices; a vertex on edge (a, b) is X_a + t (X_b
 *     - X_a), t = f_a / (f_a - f_b) clamped to [0, 1], f = sqrt(edt2) h - p.
 * Outputs (device or page-locked host memory): tris float [max_tris][3][3]
 * (A); labels (nullable) int64 [max_tris][3]: cell * 16 + edge (0..11) for
 * edge vertices, cell * 16 + 12 + loop for loop means, cell = (k (ny-1) +
 * j) (nx-1) + i; sas (nullable) uint8 and edt2 (nullable) uint16, both
 * [nz][ny][nx].  *n_tris (host) receives the total number of triangles;
 * when it exceeds max_tris only the first max_tris are written and the call
 * returns VTX_ERR_CAPACITY.  Scratch (8 bytes per grid point) is owned by
 * the context.  Synchronises.
 */
vtx_status vtx_ses_mesh(vtx_ctx *ctx, const float *xyzr, int64_t n_atoms, const vtx_ses_grid *grid, float *tris,
                        int64_t max_tris, int64_t *labels, uint8_t *sas, uint16_t *edt2, int64_t *n_tris);

/* Synchronise the context's stream and report (once) any device-side error. */
vtx_status vtx_sync_status(vtx_ctx *ctx);

/*
 * Per-stage GPU times (ms), averaged over every pipeline run made with
 * VTX_FLAG_PROFILE or VTX_FLAG_PROFILE_CULL since the previous call, measured with CUDA events
 * recorded on the context's stream between the stages (clear, cull, setup,
 * scan, scatter, raster, resolve: background pixels and the covered-pixel
 * list, shade: the covered pixels' hit, shading, SSAO and post-processing;
 * with a single-pass resolve "shade" is 0).  Runs made with
 * VTX_FLAG_PROFILE_CULL (and not VTX_FLAG_PROFILE) contribute to the cull's
 * average only; a stage no run measured reports 0.  names/ms: arrays of *n
 * entries (in: capacity; out: stages written); *runs (may be NULL) receives
 * the number of profiled runs.  Waits for the last profiled run, then
 * forgets the runs.
 */
vtx_status vtx_stage_times(vtx_ctx *ctx, const char **names, float *ms, int32_t *n, int32_t *runs);

/*
 * The tile shape and direct-splat threshold chosen by the autotuner for the
 * most recent render call made with settings.tile_w = 0.  The tuner times all
 * nine combinations of tile shape (16x16, 32x8, 8x8) and threshold (4, 16, 64
 * candidate pixels) on the caller's own frame (a batch: its first four
 * frames) once per class (image size, views, log2 of the primitive count,
 * mode) and reuses the fastest.  The output never depends on the choice.
 * Returns VTX_ERR_STATE before any tuned call.
 */
vtx_status vtx_tuned_settings(const vtx_ctx *ctx, int32_t *tile_w, int32_t *tile_h, int32_t *splat_max_px);

/*
 * Failure-injection hooks for tests of the error paths (the paper has no
 * counterpart).  Every hook acts on the host side or bounds a device wait,
 * so none of them can fault or hang the GPU:
 *   first_wait_polls >= 0: the multi-view / batch cull gives its FIRST
 *     bulk-copy wait only that many polls (0: it gives up at once), sets the
 *     timeout bit and stops; its drain of copies in flight keeps the normal
 *     limit.  The next synchronising call reports VTX_ERR_TIMEOUT.  -1
 *     restores the normal limit.
 *   cap_records, cap_entries > 0: set the scratch arena's record and
 *     tile-entry capacities (smaller capacities overflow; the next
 *     synchronising call reports VTX_ERR_CAPACITY once and grows them).
 *   corrupt_key != 0: after the tile ray-cast, pixel (0, 0)'s depth key is
 *     overwritten by a host memset with an out-of-range primitive id; the
 *     resolve's bounds check draws it as background and the next
 *     synchronising call reports VTX_ERR_BOUNDS.  0 turns it off.
 * Hooks persist on the context until changed.  Cached batch graphs are
 * dropped.
 */
vtx_status vtx_debug_hooks(vtx_ctx *ctx, int32_t first_wait_polls, uint32_t cap_records, uint64_t cap_entries,
                           int32_t corrupt_key);

/*
 * Text of the most recent error on this context ("" if none; "null context"
 * for NULL).  The engine's log of failures (the paper's console of logs,
 * Figure 1) reduced to the last message; the pointer stays valid until the
 * next call on the context.
 */
const char *vtx_last_error(const vtx_ctx *ctx);

/*
 * Measurement helper, with no counterpart in the paper: the FP32
 * multiply-add rate of the current device, the denominator of the rooflines
 * of the compute-bound kernels (tile ray-cast, soft forward and backward).
 * Runs 8 blocks of 256 threads per SM, each thread with 8 independent FMA
 * chains of `iters` x 16 steps, once untimed and once timed with CUDA events
 * on cuda_stream (NULL = default); paired != 0 issues them as paired FFMA2
 * instructions, 0 as scalar FFMA (whose rate / 64 is also the warp
 * instruction issue rate).  *ms receives the timed launch's duration and
 * *flops its floating-point operations (2 per FMA).  Allocates and frees 4
 * bytes of device memory; synchronises.  Clocks are left as they are.
 */
vtx_status vtx_measure_fp32_rate(int32_t paired, int32_t iters, void *cuda_stream, float *ms, double *flops);

/*
 * Allocation-free visibility buffer.  The paper has no counterpart: this
 * entry point exists for callers that cannot allocate device memory (code
 * running inside an allocator or memory-pool callback, plug-ins of an
 * application that owns every allocation on the device, real-time loops
 * that must not trigger cudaMalloc's implicit synchronisation).  It renders
 * the nearest atom id and its depth per pixel for van der Waals spheres
 * (the same ids and depths as vtx_render_frame) using scratch held in a
 * file-scope __device__ array of VTX_STATIC_MAX_PIXELS 64-bit depth keys
 * (8 MiB, kept by every GPU that loads the library until the process exits).
 * No cudaMalloc, cudaFree or other allocating routine is called.
 *   xyzr: device float4 [n_atoms] (16-byte aligned); cam: host camera with
 *   width*height <= VTX_STATIC_MAX_PIXELS; depth: device float [H][W]
 *   (+inf for background); id: device uint32 [H][W] (0xFFFFFFFF for
 *   background); cuda_stream: the stream to enqueue on (NULL = default).
 * Returns VTX_ERR_CAPACITY for larger images, VTX_ERR_INVALID_ARG for bad
 * arguments, VTX_ERR_CUDA if a launch fails.  Work is only enqueued.
 * The first call on a device looks up the array's device address with that
 * device current (cudaGetSymbolAddress), so make that first call before any
 * stream capture.  Every call shares the one array and clears it first:
 * calls whose work overlaps on the GPU (other streams, other threads) race
 * on it and must be serialised by the caller.
 */
#define VTX_STATIC_MAX_PIXELS (1 << 20)
vtx_status vtx_render_visibility_static(const float *xyzr, int64_t n_atoms, const vtx_camera *cam, float *depth,
                                        uint32_t *id, void *cuda_stream);

#ifdef __cplusplus
}
#endif

#endif /* VTX_H_ */
