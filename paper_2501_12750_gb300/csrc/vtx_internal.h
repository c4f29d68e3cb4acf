// vtx_internal.h -- host-side declarations shared by the renderer's translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/vtx.h"
#include "vtx_device.cuh"

namespace vtx {

#ifndef VTX_OCCL_PIXELS
#define VTX_OCCL_PIXELS 4
#endif
constexpr long long kOcclPixels = VTX_OCCL_PIXELS;  // occlusion pass from one survivor per this many pixels

// Tile counts that the one-CTA scan covers (32 warps x 32 lanes x 32 values); more take the three-kernel scan,
// whose tile list is unordered and holds the non-empty tiles only.
constexpr long long kScanSingleMax = 32LL * 32 * 32;

// Device buffers of one pipeline run (all owned by the context).
struct Scratch {
  unsigned long long *keys;   // [n_img][H][W] packed (depth key << 32 | id)
  uint32_t *surv;             // [n_img][surv_cap] survivor primitive ids
  ImageState *state;          // [n_img]
  uint32_t *tile_count;       // [n_tiles]
  uint32_t *tile_start;       // [n_tiles + 1] exclusive prefix (tile_start[n_tiles] = total, clamped)
  uint32_t *tile_cursor;      // [n_tiles]
  uint32_t *block_sums;       // [ceil(n_tiles / 4096) + 1]
  uint32_t *tile_list;        // [n_tiles] indices of the non-empty tiles, longest list first (one-CTA scan);
                              // the soft path's one-CTA scan lists the empty tiles after them
  PrimRec *recs;              // [cap_rec]
  uint32_t *rec_img;          // [cap_rec] image of each record
  uint2 *rec_box;             // [cap_rec] tile box of each record: (x0 | y0 << 16, x1 | y1 << 16)
  uint32_t *rec_of;           // soft: [n_img][n_atoms] record of each atom
  unsigned long long *entries;  // [cap_entries] (sort key << 32 | record or id)
  uint32_t *cov_list;         // [n_img * H * W] covered pixels (img * H * W + p), or null: single-pass resolve
  uint32_t *cov_mask;         // [n_img * H * W / 32 + 8] coverage bits written by the list pass
  uint32_t *defer;            // occlusion pass: [n_img][surv_cap] the survivors its test kept, or null
  Status *status;
  uint32_t cap_rec;
  unsigned long long cap_entries;
};

struct Scene {
  const float4 *frames;       // [n_frames][stride]
  const long long *counts;    // device [n_frames] atom counts, or null (all = n_atoms)
  const uint8_t *elem;        // [stride] or null
  const uint2 *bonds;         // [n_bonds] or null
  float4 *stage;              // single view, no bonds: device copy of the surviving records, written by the cull
                              // and read by setup and resolve instead of frames (frames in host memory), or null
  bool dbg_corrupt_key = false;  // test hook: overwrite the first depth key with an out-of-range id after the raster
};

struct Outputs {
  float *depth;
  uint32_t *id;
  float *normal;
  float *rgb;
  float *ao;
};

struct StageEvents {
  cudaEvent_t *ev;  // array of events, one recorded after each stage (may be null)
  int n;
  unsigned mask = ~0u;  // bit i set: record event i
};

// Hard-edge pipeline: cull .. resolve.  Returns the first launch error.
cudaError_t run_frame_pipeline(const Geometry &g, const ShadeParams &sh, const Scene &sc, const Scratch &s,
                               const Outputs &out, bool ssao, cudaStream_t st, StageEvents *evs);

// Soft-edge pipeline (binning shared with the hard path); backward when grad != null.
// state: optional per-pixel (final transmittance, 1 + last contributor) planes, written by the forward
// call and read by the backward call (which then skips its front-to-back walk).
// reuse_lists (backward only): the scratch still holds the tile lists, records and tile order that the
// forward call on the same inputs built and ordered; the backward skips the binning and the sort.
cudaError_t run_soft_pipeline(const Geometry &g, const Scene &sc, const Scratch &s, float *cov, float *depth,
                              float *normal, const float *g_cov, const float *g_depth, const float *g_normal,
                              float *grad, uint2 *state, bool reuse_lists, cudaStream_t st, StageEvents *evs);

// Interleaved RGBA8 of n_img images of ppi pixels from the rgb and id planes (background alpha bg_a).
cudaError_t run_export_rgba8(const float *rgb, const uint32_t *id, long long ppi, long long n_img, unsigned char bg_a,
                             uint8_t *rgba, cudaStream_t st);

// Solvent excluded surface on a grid (ses.cu).
struct SesLaunch {
  const float4 *X;
  long long n_atoms;
  float origin[3];
  float h, probe;
  int32_t dims[3];
  uint8_t *sas;                   // [nz][ny][nx] SAS interior (0/1)
  uint16_t *g_a, *g_b;            // distance-pass scratch, one value per grid point each
  uint16_t *edt2;                 // [nz][ny][nx] windowed squared distance (grid units)
  uint8_t *cases;                 // [(nz-1)(ny-1)(nx-1)] marching-cubes case of every cell
  unsigned *block_tris;           // [ses_blocks(dims)]
  unsigned long long *block_base; // [ses_blocks(dims)]
  unsigned long long *total;      // [1]
  float *tris;                    // [max_tris][3][3]
  long long *labels;              // [max_tris][3] or null
  long long max_tris;
};
cudaError_t run_ses_grid(const SesLaunch &L, cudaStream_t st);
cudaError_t run_ses_bbox(const float4 *X, long long n, float probe, float *partial, int n_blocks, cudaStream_t st);
long long ses_blocks(const int32_t dims[3]);
int ses_window(float probe, float h);

int sm_count();

// Per-camera constants of the kernels (FP64-derived focal length, cull margins) and the host-side camera check
// (sizes 1..16384, finite eye and basis, finite tan_half_fovy > 0 and znear > 0), shared by every entry point.
ViewParams make_view(const vtx_camera &cam);
bool cam_ok(const vtx_camera *c);

// Extra survivor slots the single-view cull may leave as holes (per-warp slabs).
long long cull_survivor_slack(long long n_atoms);
// The same for each image of the multi-view batch cull (per_frame: atom slots per frame).
long long cull_multi_slack(long long per_frame, int n_frames);

}  // namespace vtx
