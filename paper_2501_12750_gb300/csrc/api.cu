// api.cu -- C ABI of the renderer (declared in include/vtx.h): context,
// scratch arena, argument checks, per-frame / batched / soft entry points,
// CUDA-graph capture of batches and per-stage CUDA-event profiling.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/vtx.h"
#include "vtx_internal.h"

using namespace vtx;

namespace {

struct Buf {
  void *p = nullptr;
  size_t bytes = 0;
};

struct GraphEntry {
  std::vector<unsigned char> key;
  cudaGraphExec_t exec = nullptr;
  long long *d_counts = nullptr;
};

constexpr int kNumStages = 8;
const char *kStageNames[kNumStages] = {"clear", "cull", "setup", "scan", "scatter", "raster", "resolve", "shade"};

}  // namespace

struct vtx_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  // scene
  const float4 *xyzr = nullptr;
  bool atoms_on_host = false;  // xyzr is page-locked host memory (read over the host link)
  const uint8_t *elem = nullptr;
  long long n_atoms = 0;
  float palette[kMaxElem][3];
  int n_elem = 1;
  const uint2 *bonds = nullptr;
  long long n_bonds = 0;
  vtx_camera cam;
  bool has_cam = false;
  // scratch
  Buf keys, surv, state, tcount, tstart, tcursor, tlist, bsums, recs, recimg, recbox, recof, entries, status, counts, hostin_x,
      hostin_e, hostout, covlist, covmask, stage, defer;
  bool cov_ok = false;  // the covered-pixel list of the last prepared launch fits (two-pass resolve)
  bool occl_ok = false;  // the occlusion pass's buffers of the last prepared launch fit
  Buf ses_sas, ses_a, ses_b, ses_edt, ses_blk, ses_base, ses_total, ses_bbox, ses_case;
  uint32_t cap_rec = 0;
  unsigned long long cap_entries = 0;
  Status *h_status = nullptr;
  long long *h_counts = nullptr;
  int h_counts_cap = 0;
  cudaEvent_t counts_done = nullptr;
  // profiling: one set of 8 events per profiled pipeline run since the last read
  std::vector<cudaEvent_t *> ev_sets;
  std::vector<unsigned> ev_masks;  // per used set: the stage events it recorded
  size_t ev_used = 0;
  // graphs
  std::vector<GraphEntry> graphs;
  // autotuning results: key -> (tile_w, tile_h, splat_max)
  struct Tune {
    long long key[6];
    int tw, th, splat;
  };
  std::vector<Tune> tunes;
  int last_tw = 0, last_th = 0, last_splat = 0;
  long long soft_sized[4] = {-1, -1, -1, -1};  // (atoms, views, W, H) of the last soft run that synchronised cleanly
  // every run that sizes or replays the arena takes a new generation; a soft forward records the generation
  // and inputs of the tile lists it leaves behind, which a backward call may then reuse
  uint64_t arena_gen = 0;
  uint64_t alloc_gen = 0;  // bumped by every (re)allocation of a context buffer
  struct SoftLists {
    uint64_t gen = ~0ull;
    const float *xyzr = nullptr;
    int64_t n = 0;
    float sigma = 0.0f;
    std::vector<vtx_camera> cams;
  } soft_lists;
  // failure-injection hooks (vtx_debug_hooks)
  int dbg_first_wait = -1;
  bool dbg_corrupt_key = false;
  // output planes last checked by visible_outputs (caller pointers -> device-visible aliases)
  vtx_outputs out_in{}, out_dev{};
  std::string err;
};

static vtx_status fail(vtx_ctx *c, vtx_status s, const std::string &msg) {
  if (c) c->err = msg;
  return s;
}

static vtx_status cuda_fail(vtx_ctx *c, cudaError_t e, const char *where) {
  return fail(c, VTX_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

static vtx_status ensure(vtx_ctx *c, Buf &b, size_t bytes, const char *what) {
  if (bytes == 0) bytes = 16;
  if (b.bytes >= bytes) return VTX_OK;
  if (b.p) cudaFree(b.p);
  b.p = nullptr;
  b.bytes = 0;
  size_t want = bytes + bytes / 8;
  ++c->alloc_gen;
  cudaError_t e = cudaMalloc(&b.p, want);
  if (e != cudaSuccess) {
    cudaGetLastError();
    e = cudaMalloc(&b.p, bytes);
    if (e != cudaSuccess) {
      cudaGetLastError();
      b.p = nullptr;
      return fail(c, VTX_ERR_OOM, std::string("cudaMalloc failed for ") + what);
    }
    want = bytes;
  }
  b.bytes = want;
  return VTX_OK;
}

static void drop_graphs(vtx_ctx *c) {
  for (auto &g : c->graphs) {
    if (g.exec) cudaGraphExecDestroy(g.exec);
    if (g.d_counts) cudaFree(g.d_counts);
  }
  c->graphs.clear();
}

namespace vtx {
ViewParams make_view(const vtx_camera &cam) {
  ViewParams v;
  for (int k = 0; k < 3; ++k) {
    v.eye[k] = cam.eye[k];
    v.R[k] = cam.right[k];
    v.U[k] = cam.up[k];
    v.F[k] = cam.forward[k];
  }
  double f = (double)cam.height / (2.0 * (double)cam.tan_half_fovy);
  v.f_hi = (float)f;
  v.f_lo = (float)(f - (double)v.f_hi);
  v.f = v.f_hi;
  v.inv_f = (float)(1.0 / f);
  v.cx = 0.5f * (float)cam.width;
  v.cy = 0.5f * (float)cam.height;
  v.znear = cam.znear;
  v.pad0 = 0.0f;
  v.hc = (float)(f * (1.0 + 4e-6));
  v.e0 = (float)(1e-4 + 1e-6 * ((double)cam.width + (double)cam.height));
  v.cxm = v.cx - 0.5f;
  v.cym = v.cy - 0.5f;
  v.wm1 = (float)(cam.width - 1);
  v.hm1 = (float)(cam.height - 1);
  return v;
}

bool cam_ok(const vtx_camera *c) {
  if (!c) return false;
  if (c->width < 1 || c->height < 1 || c->width > 16384 || c->height > 16384) return false;
  if (!(c->tan_half_fovy > 0.0f) || !std::isfinite(c->tan_half_fovy)) return false;
  if (!(c->znear > 0.0f) || !std::isfinite(c->znear)) return false;
  for (int k = 0; k < 3; ++k)
    if (!std::isfinite(c->eye[k]) || !std::isfinite(c->forward[k]) || !std::isfinite(c->right[k]) ||
        !std::isfinite(c->up[k]))
      return false;
  return true;
}
}  // namespace vtx

static vtx_status settings_ok(vtx_ctx *c, const vtx_settings *s) {
  if (!s) return fail(c, VTX_ERR_INVALID_ARG, "settings is NULL");
  if (s->mode < VTX_MODE_VDW || s->mode > VTX_MODE_SAS) return fail(c, VTX_ERR_INVALID_ARG, "bad mode");
  if (s->shading < VTX_SHADE_GLOSSY || s->shading > VTX_SHADE_TOON) return fail(c, VTX_ERR_INVALID_ARG, "bad shading");
  if (s->shading == VTX_SHADE_TOON && (s->toon_levels < 2 || s->toon_levels > 16))
    return fail(c, VTX_ERR_INVALID_ARG, "toon_levels must be 2..16");
  if (!(s->fog_density >= 0.0f && s->fog_density <= 1.0f)) return fail(c, VTX_ERR_INVALID_ARG, "fog_density");
  if (!(s->outline_depth >= 0.0f)) return fail(c, VTX_ERR_INVALID_ARG, "outline_depth");
  if (s->mode == VTX_MODE_SAS && !(s->probe_radius >= 0.0f)) return fail(c, VTX_ERR_INVALID_ARG, "probe_radius");
  if (s->ssao_samples < 0 || s->ssao_samples > VTX_MAX_SSAO_SAMPLES)
    return fail(c, VTX_ERR_INVALID_ARG, "ssao_samples out of range");
  if (s->tile_w != 0) {
    int tw = s->tile_w, th = s->tile_h;
    if (!((tw == 16 && th == 16) || (tw == 32 && th == 8) || (tw == 8 && th == 8)))
      return fail(c, VTX_ERR_INVALID_ARG, "unsupported tile size");
  }
  if (s->splat_max_px < 0) return fail(c, VTX_ERR_INVALID_ARG, "splat_max_px < 0");
  if ((s->mode == VTX_MODE_BALL_AND_STICK || s->mode == VTX_MODE_STICKS) &&
      (!(s->ball_radius >= 0.0f) || !(s->bond_radius > 0.0f)))
    return fail(c, VTX_ERR_INVALID_ARG, "ball-and-stick radii");
  return VTX_OK;
}

static ShadeParams make_shade(const vtx_ctx *c, const vtx_settings *s) {
  ShadeParams sh;
  memset(&sh, 0, sizeof(sh));
  sh.model = s->shading;
  sh.toon_levels = s->toon_levels;
  sh.fog_near = s->fog_near;
  sh.fog_far = s->fog_far;
  sh.fog_density = s->fog_density;
  sh.outline_depth = s->outline_depth;
  for (int k = 0; k < 3; ++k) sh.outline_color[k] = s->outline_color[k];
  sh.ka = s->ka;
  sh.kd = s->kd;
  sh.ks = s->ks;
  sh.shin = s->shininess;
  double L[3] = {s->light_dir[0], s->light_dir[1], s->light_dir[2]};
  double ln = std::sqrt(L[0] * L[0] + L[1] * L[1] + L[2] * L[2]);
  if (!(ln > 0.0)) ln = 1.0;
  for (int k = 0; k < 3; ++k) {
    sh.L[k] = (float)(L[k] / ln);
    sh.bg[k] = s->background[k];
  }
  for (int e = 0; e < kMaxElem; ++e)
    for (int k = 0; k < 3; ++k) sh.palette[e][k] = c->palette[e][k];
  sh.n_elem = c->n_elem;
  sh.ssao_n = (s->flags & VTX_FLAG_NO_SSAO) ? 0 : s->ssao_samples;
  sh.ssao_radius = s->ssao_radius;
  sh.ssao_bias = s->ssao_bias;
  for (int j = 0; j < VTX_MAX_SSAO_SAMPLES; ++j)
    for (int k = 0; k < 3; ++k) sh.kernel[j][k] = s->ssao_kernel[j][k];
  return sh;
}

static void base_geometry(Geometry &g, const vtx_camera *cams, int n_views, int tile_w, int tile_h) {
  memset(&g, 0, sizeof(g));
  for (int v = 0; v < n_views; ++v) g.views[v] = make_view(cams[v]);
  g.n_views = n_views;
  g.W = cams[0].width;
  g.H = cams[0].height;
  g.tile_w = tile_w;
  g.tile_h = tile_h;
  g.tiles_x = (g.W + tile_w - 1) / tile_w;
  g.tiles_y = (g.H + tile_h - 1) / tile_h;
  g.tiles_per_img = g.tiles_x * g.tiles_y;
  g.pix_per_img = (long long)g.W * g.H;
  g.dbg_first_wait = -1;
}

// Size the arena for a launch; records/entries grow only through overflow reports.
static vtx_status prepare(vtx_ctx *c, const Geometry &g, bool soft, long long stride_for_recof) {
  ++c->arena_gen;
  const long long n_img = g.n_img;
  const long long n_tiles = n_img * g.tiles_per_img;
  vtx_status st;
  if (!soft && (st = ensure(c, c->keys, sizeof(unsigned long long) * (size_t)(n_img * g.pix_per_img), "keys")))
    return st;
  if ((st = ensure(c, c->surv, sizeof(uint32_t) * (size_t)(n_img * g.surv_cap), "survivors"))) return st;
  if ((st = ensure(c, c->state, sizeof(ImageState) * (size_t)n_img, "image state"))) return st;
  if ((st = ensure(c, c->tcount, sizeof(uint32_t) * (size_t)(n_tiles + 1), "tile counts"))) return st;
  if ((st = ensure(c, c->tstart, sizeof(uint32_t) * (size_t)(n_tiles + 1), "tile starts"))) return st;
  if ((st = ensure(c, c->tcursor, sizeof(uint32_t) * (size_t)(n_tiles + 1), "tile cursors"))) return st;
  if ((st = ensure(c, c->tlist, sizeof(uint32_t) * (size_t)(n_tiles + 1), "tile list"))) return st;
  if ((st = ensure(c, c->bsums, sizeof(unsigned long long) * (size_t)(n_tiles / 4096 + 4), "scan blocks"))) return st;
  if (c->cap_rec == 0) {
    long long est = n_img * g.stride / 8;
    est = est < (1 << 16) ? (1 << 16) : (est > (1 << 22) ? (1 << 22) : est);
    c->cap_rec = (uint32_t)est;
    c->cap_entries = 4ull * est;
  }
  if ((st = ensure(c, c->recs, sizeof(PrimRec) * (size_t)c->cap_rec, "records"))) return st;
  if ((st = ensure(c, c->recimg, sizeof(uint32_t) * (size_t)c->cap_rec, "record images"))) return st;
  if ((st = ensure(c, c->recbox, sizeof(uint2) * (size_t)c->cap_rec, "record boxes"))) return st;
  if ((st = ensure(c, c->entries, sizeof(unsigned long long) * (size_t)c->cap_entries, "entries"))) return st;
  if (soft &&(st = ensure(c, c->recof, sizeof(uint32_t) * (size_t)(n_img * stride_for_recof), "record map")))
    return st;
  if (!c->status.p) {
    if ((st = ensure(c, c->status, sizeof(Status), "status"))) return st;
    cudaMemsetAsync(c->status.p, 0, sizeof(Status), c->stream);
  }
  // occlusion pass: the kept survivors' list (no room: the plain setup does without)
  c->occl_ok = false;
  if (g.occl && !soft) {
    if (ensure(c, c->defer, sizeof(uint32_t) * (size_t)(n_img * g.surv_cap), "kept survivors") == VTX_OK)
      c->occl_ok = true;
    else
      c->err.clear();
  }
  // covered-pixel list of the two-pass resolve (32-bit entries: only when every pixel index fits)
  c->cov_ok = false;
  if (!soft && n_img * g.pix_per_img < 4294967295LL) {
    if (ensure(c, c->covlist, sizeof(uint32_t) * (size_t)(n_img * g.pix_per_img), "covered pixels") == VTX_OK &&
        ensure(c, c->covmask, sizeof(uint32_t) * (size_t)(n_img * g.pix_per_img / 32 + 8), "coverage bits") == VTX_OK)
      c->cov_ok = true;
    else
      c->err.clear();  // no room: the single-pass resolve needs no list
  }
  return VTX_OK;
}

static Scratch scratch_of(vtx_ctx *c) {
  Scratch s;
  s.keys = (unsigned long long *)c->keys.p;
  s.surv = (uint32_t *)c->surv.p;
  s.state = (ImageState *)c->state.p;
  s.tile_count = (uint32_t *)c->tcount.p;
  s.tile_start = (uint32_t *)c->tstart.p;
  s.tile_cursor = (uint32_t *)c->tcursor.p;
  s.block_sums = (uint32_t *)c->bsums.p;
  s.tile_list = (uint32_t *)c->tlist.p;
  s.recs = (PrimRec *)c->recs.p;
  s.rec_img = (uint32_t *)c->recimg.p;
  s.rec_box = (uint2 *)c->recbox.p;
  s.rec_of = (uint32_t *)c->recof.p;
  s.entries = (unsigned long long *)c->entries.p;
  s.status = (Status *)c->status.p;
  s.cap_rec = c->cap_rec;
  s.cap_entries = c->cap_entries;
  s.cov_list = c->cov_ok ? (uint32_t *)c->covlist.p : nullptr;
  s.cov_mask = c->cov_ok ? (uint32_t *)c->covmask.p : nullptr;
  s.defer = c->occl_ok ? (uint32_t *)c->defer.p : nullptr;
  return s;
}

// Read the device status; on overflow grow the arena and clear the flags.
static vtx_status check_status(vtx_ctx *c) {
  cudaError_t e = cudaMemcpyAsync(c->h_status, c->status.p, sizeof(Status), cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "device error");
  Status s = *c->h_status;
  if (s.overflow == 0u) return VTX_OK;
  if (s.overflow & 16u) {
    cudaMemsetAsync(c->status.p, 0, sizeof(Status), c->stream);
    return fail(c, VTX_ERR_TIMEOUT, "a device-side wait for a bulk copy gave up; the frame is invalid");
  }
  if (s.overflow & 32u) {
    cudaMemsetAsync(c->status.p, 0, sizeof(Status), c->stream);
    return fail(c, VTX_ERR_BOUNDS, "a decoded primitive id was out of range (drawn as background); the frame is invalid");
  }
  std::string msg = "scratch capacity exceeded:";
  unsigned long long need_e = s.n_entries;
  if (s.overflow & 2u) {
    const unsigned long long written = c->cap_rec > 0 ? c->cap_rec : 1;
    unsigned long long need = (unsigned long long)s.n_rec;
    unsigned long long cap = need + need / 2 + 1024;
    if (cap > 0xfffffff0ull) cap = 0xfffffff0ull;
    if (cap > c->cap_rec) c->cap_rec = (uint32_t)cap;
    // the tile entries were counted from the records that fitted only: scale them to all records, so one
    // re-render suffices
    if (need > written) need_e = (unsigned long long)((double)need_e * (double)need / (double)written);
    msg += " records";
  }
  if ((s.overflow & 4u) || need_e > c->cap_entries) {
    unsigned long long cap = need_e + need_e / 2 + 4096;
    if (cap > 0xfffffff0ull) cap = 0xfffffff0ull;
    if (cap > c->cap_entries) c->cap_entries = cap;
    msg += " tile entries";
  }
  cudaMemsetAsync(c->status.p, 0, sizeof(Status), c->stream);
  drop_graphs(c);
  vtx_status st;
  if ((st = ensure(c, c->recs, sizeof(PrimRec) * (size_t)c->cap_rec, "records"))) return st;
  if ((st = ensure(c, c->recimg, sizeof(uint32_t) * (size_t)c->cap_rec, "record images"))) return st;
  if ((st = ensure(c, c->recbox, sizeof(uint2) * (size_t)c->cap_rec, "record boxes"))) return st;
  if ((st = ensure(c, c->entries, sizeof(unsigned long long) * (size_t)c->cap_entries, "entries"))) return st;
  return fail(c, VTX_ERR_CAPACITY, msg + " (arena grown; render again)");
}

// Events for one profiled render.  VTX_FLAG_PROFILE: a start event and one
// after every stage.  VTX_FLAG_PROFILE_CULL: only the events after the clear
// and after the cull (the cull's duration is their difference).
static StageEvents *events_for(vtx_ctx *c, const vtx_settings *s, StageEvents &ev) {
  if (!(s && (s->flags & (VTX_FLAG_PROFILE | VTX_FLAG_PROFILE_CULL)))) return nullptr;
  if (c->ev_used == c->ev_sets.size()) {
    cudaEvent_t *set = new cudaEvent_t[kNumStages + 1];
    for (int i = 0; i <= kNumStages; ++i) cudaEventCreate(&set[i]);
    c->ev_sets.push_back(set);
    c->ev_masks.push_back(0u);
  }
  const size_t r = c->ev_used++;
  cudaEvent_t *set = c->ev_sets[r];
  const bool full = (s->flags & VTX_FLAG_PROFILE) != 0;
  c->ev_masks[r] = full ? ~0u : 3u;
  if (full) cudaEventRecord(set[kNumStages], c->stream);  // start
  ev.ev = set;
  ev.n = kNumStages;
  ev.mask = c->ev_masks[r];
  return &ev;
}

extern "C" {

const char *vtx_version(void) { return "vtx-gb300 0.1 (sm_103a)"; }

vtx_status vtx_default_settings(vtx_settings *s) {
  if (!s) return VTX_ERR_INVALID_ARG;
  memset(s, 0, sizeof(*s));
  s->mode = VTX_MODE_VDW;
  s->ball_radius = 0.4f;
  s->bond_radius = 0.15f;
  s->ka = 0.2f;
  s->kd = 0.7f;
  s->ks = 0.3f;
  s->shininess = 32.0f;
  s->light_dir[0] = 0.25f;
  s->light_dir[1] = 0.5f;
  s->light_dir[2] = 1.0f;
  s->background[0] = s->background[1] = s->background[2] = 1.0f;
  s->ssao_samples = 0;
  s->ssao_radius = 2.0f;
  s->ssao_bias = 0.025f;
  s->tile_w = 16;
  s->tile_h = 16;
  s->splat_max_px = 0;  // the library default: by primitives per pixel
  s->shading = VTX_SHADE_GLOSSY;
  s->toon_levels = 4;
  s->probe_radius = 1.4f;
  s->fog_near = 0.0f;
  s->fog_far = 0.0f;
  s->fog_density = 0.0f;
  s->outline_depth = 0.0f;
  return VTX_OK;
}

vtx_status vtx_create(vtx_ctx **out, int32_t device, void *cuda_stream) {
  if (!out) return VTX_ERR_INVALID_ARG;
  *out = nullptr;
  int n = 0;
  if (cudaGetDeviceCount(&n) != cudaSuccess || device < 0 || device >= n) {
    cudaGetLastError();
    return VTX_ERR_INVALID_ARG;
  }
  vtx_ctx *c = new vtx_ctx();
  c->device = device;
  cudaSetDevice(device);
  c->stream = (cudaStream_t)cuda_stream;
  for (int e = 0; e < kMaxElem; ++e) c->palette[e][0] = c->palette[e][1] = c->palette[e][2] = 0.5f;
  if (cudaMallocHost((void **)&c->h_status, sizeof(Status)) != cudaSuccess) {
    cudaGetLastError();
    delete c;
    return VTX_ERR_OOM;
  }
  memset(c->h_status, 0, sizeof(Status));
  cudaEventCreateWithFlags(&c->counts_done, cudaEventDisableTiming);
  *out = c;
  return VTX_OK;
}

vtx_status vtx_destroy(vtx_ctx *c) {
  if (!c) return VTX_ERR_INVALID_ARG;
  cudaSetDevice(c->device);
  cudaStreamSynchronize(c->stream);
  drop_graphs(c);
  Buf *bufs[] = {&c->keys,   &c->surv,   &c->state,  &c->tcount,   &c->tstart,   &c->tcursor,  &c->tlist,
                 &c->bsums,  &c->recs,   &c->recimg, &c->recbox,   &c->recof,    &c->entries,  &c->status,
                 &c->counts, &c->hostin_x, &c->hostin_e, &c->hostout, &c->covlist, &c->covmask, &c->stage, &c->defer, &c->ses_sas, &c->ses_a, &c->ses_b,
                 &c->ses_edt, &c->ses_blk, &c->ses_base, &c->ses_total, &c->ses_bbox, &c->ses_case};
  for (Buf *b : bufs)
    if (b->p) cudaFree(b->p);
  if (c->h_status) cudaFreeHost(c->h_status);
  if (c->h_counts) cudaFreeHost(c->h_counts);
  if (c->counts_done) cudaEventDestroy(c->counts_done);
  for (cudaEvent_t *set : c->ev_sets) {
    for (int i = 0; i <= kNumStages; ++i) cudaEventDestroy(set[i]);
    delete[] set;
  }
  delete c;
  return VTX_OK;
}

vtx_status vtx_set_stream(vtx_ctx *c, void *cuda_stream) {
  if (!c) return VTX_ERR_INVALID_ARG;
  c->stream = (cudaStream_t)cuda_stream;
  drop_graphs(c);
  return VTX_OK;
}

// Device-visible address of a caller array: device or managed memory as is,
// page-locked host memory through its mapped alias (the kernels then read it
// over the host link, so it never has to fit in device memory).  Pageable
// host memory is refused rather than relying on the platform's support for
// device access to it.
static bool device_visible(vtx_ctx *c, const void *p, const void **dev, const char *what, bool *on_host = nullptr) {
  *dev = p;
  if (on_host) *on_host = false;
  if (!p) return true;
  cudaPointerAttributes a;
  cudaError_t e = cudaPointerGetAttributes(&a, p);
  if (e != cudaSuccess) {
    cudaGetLastError();
    fail(c, VTX_ERR_INVALID_ARG, what);
    return false;
  }
  if (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged) return true;
  if (a.type == cudaMemoryTypeHost && a.devicePointer) {
    *dev = a.devicePointer;
    if (on_host) *on_host = true;
    return true;
  }
  fail(c, VTX_ERR_INVALID_ARG, what);
  return false;
}

// Output planes as the kernels address them: device memory as is, page-locked
// host planes through their mapped aliases (the resolve then writes them over
// the host link).  The last translation is cached per context.
static vtx_status visible_outputs(vtx_ctx *c, const vtx_outputs *in, vtx_outputs *dev) {
  if (memcmp(in, &c->out_in, sizeof(vtx_outputs)) == 0 && c->out_dev.depth) {
    *dev = c->out_dev;
    return VTX_OK;
  }
  const void *d[5];
  const void *src[5] = {in->depth, in->id, in->normal, in->rgb, in->ao};
  for (int k = 0; k < 5; ++k)
    if (!device_visible(c, src[k], &d[k], "outputs: not device memory or page-locked host memory"))
      return VTX_ERR_INVALID_ARG;
  dev->depth = (float *)d[0];
  dev->id = (uint32_t *)d[1];
  dev->normal = (float *)d[2];
  dev->rgb = (float *)d[3];
  dev->ao = (float *)d[4];
  c->out_in = *in;
  c->out_dev = *dev;
  return VTX_OK;
}

vtx_status vtx_upload_atoms(vtx_ctx *c, const float *xyzr, const uint8_t *elem, const float *palette_rgb,
                            int32_t n_elem, int64_t n_atoms) {
  if (!c) return VTX_ERR_INVALID_ARG;
  cudaSetDevice(c->device);
  if (n_atoms < 0 || n_atoms > 2147483647LL) return fail(c, VTX_ERR_INVALID_ARG, "n_atoms out of range");
  if (n_atoms > 0 && !xyzr) return fail(c, VTX_ERR_INVALID_ARG, "xyzr is NULL");
  if (((uintptr_t)xyzr & 15u) != 0) return fail(c, VTX_ERR_INVALID_ARG, "xyzr must be 16-byte aligned");
  if (n_elem < 1 || n_elem > VTX_MAX_ELEMENTS || !palette_rgb)
    return fail(c, VTX_ERR_INVALID_ARG, "palette: need 1..32 elements");
  const void *dx = nullptr, *de = nullptr;
  bool host_atoms = false;
  if (!device_visible(c, xyzr, &dx, "xyzr: not device memory or page-locked host memory", &host_atoms))
    return VTX_ERR_INVALID_ARG;
  if (!device_visible(c, elem, &de, "elem: not device memory or page-locked host memory")) return VTX_ERR_INVALID_ARG;
  if (((uintptr_t)dx & 15u) != 0) return fail(c, VTX_ERR_INVALID_ARG, "xyzr alias must be 16-byte aligned");
  c->xyzr = (const float4 *)dx;
  c->atoms_on_host = host_atoms;
  c->elem = (const uint8_t *)de;
  c->n_atoms = n_atoms;
  c->n_elem = n_elem;
  for (int e = 0; e < n_elem; ++e)
    for (int k = 0; k < 3; ++k) c->palette[e][k] = palette_rgb[3 * e + k];
  c->bonds = nullptr;
  c->n_bonds = 0;
  drop_graphs(c);
  return VTX_OK;
}

vtx_status vtx_upload_bonds(vtx_ctx *c, const uint32_t *pairs, int64_t n_bonds) {
  if (!c) return VTX_ERR_INVALID_ARG;
  if (n_bonds < 0 || c->n_atoms + n_bonds > 4294967040LL) return fail(c, VTX_ERR_INVALID_ARG, "n_bonds out of range");
  if (n_bonds > 0 && !pairs) return fail(c, VTX_ERR_INVALID_ARG, "pairs is NULL");
  if (((uintptr_t)pairs & 7u) != 0) return fail(c, VTX_ERR_INVALID_ARG, "pairs must be 8-byte aligned");
  cudaSetDevice(c->device);
  const void *dp = nullptr;
  if (n_bonds > 0 && !device_visible(c, pairs, &dp, "pairs: not device memory or page-locked host memory"))
    return VTX_ERR_INVALID_ARG;
  if (((uintptr_t)dp & 7u) != 0) return fail(c, VTX_ERR_INVALID_ARG, "pairs alias must be 8-byte aligned");
  c->bonds = n_bonds > 0 ? (const uint2 *)dp : nullptr;
  c->n_bonds = n_bonds;
  drop_graphs(c);
  return VTX_OK;
}

vtx_status vtx_set_camera(vtx_ctx *c, const vtx_camera *cam) {
  if (!c) return VTX_ERR_INVALID_ARG;
  if (!cam_ok(cam)) return fail(c, VTX_ERR_INVALID_ARG, "invalid camera");
  c->cam = *cam;
  c->has_cam = true;
  return VTX_OK;
}

static void set_representation(Geometry &g, const vtx_settings *s) {
  g.mode = s->mode;
  g.ball_radius = s->ball_radius;
  g.bond_radius = s->bond_radius;
  g.probe = s->probe_radius;
  for (int k = 0; k < 4; ++k) g.clip[k] = s->clip_plane[k];
  g.clip_on = (s->clip_plane[0] != 0.0f || s->clip_plane[1] != 0.0f || s->clip_plane[2] != 0.0f) ? 1 : 0;
}

// Library-default direct-splat threshold (splat_max_px = 0): sparse frames (at most one primitive per 8
// pixels) bin all but the smallest primitives for the tile raster (4 px), crowded ones splat boxes of up to
// 16 px directly.  Measured with the autotuner: the 1e5-atom 1080p frame is fastest at 4 (0.082 -> 0.078
// ms), the 1e8-atom 4K frame and the 500k-atom trajectory images at 16.  Every threshold gives the same planes.
static int default_splat(long long prims_per_img, long long pix_per_img) {
  return prims_per_img * 8 <= pix_per_img ? 4 : 16;
}

static vtx_status render_once(vtx_ctx *c, const vtx_settings *s, const vtx_outputs *out, StageEvents *ev) {
  Geometry g;
  int tw = s->tile_w ? s->tile_w : 16, th = s->tile_h ? s->tile_h : 16;
  base_geometry(g, &c->cam, 1, tw, th);
  g.n_frames = 1;
  g.n_img = 1;
  set_representation(g, s);
  g.soft = 0;
  g.stride = c->n_atoms;
  g.n_atoms = c->n_atoms;
  g.n_bonds = (s->mode == VTX_MODE_BALL_AND_STICK || s->mode == VTX_MODE_STICKS) ? c->n_bonds : 0;
  g.splat_max = s->splat_max_px ? s->splat_max_px : default_splat(g.n_atoms + g.n_bonds, g.pix_per_img);
  g.surv_cap = c->n_atoms + g.n_bonds + cull_survivor_slack(c->n_atoms);
  // no occlusion pass for a single frame: measured on the 1e8-atom 4K frame (whose set-up is 0.07 ms of
  // 0.43) it cost more than it saved (2,331 -> 1,959 frames/s, with the bounds then in a plane of their own):
  // its two passes over every survivor outweigh the set-up they remove
  g.occl = 0;
  vtx_status st = prepare(c, g, false, 0);
  if (st) return st;
  g.dbg_first_wait = c->dbg_first_wait;
  Scene sc{c->xyzr, nullptr, c->elem, g.n_bonds ? c->bonds : nullptr, nullptr};
  sc.dbg_corrupt_key = c->dbg_corrupt_key;
  // host-resident atoms: the cull copies its survivors into device memory (when there is room), so setup and
  // resolve gather them from HBM instead of over the host link (bonds need their end atoms: not staged)
  if (c->atoms_on_host && g.n_bonds == 0 && c->n_atoms > 0) {
    if (ensure(c, c->stage, sizeof(float4) * (size_t)c->n_atoms, "staged survivors") == VTX_OK)
      sc.stage = (float4 *)c->stage.p;
    else
      c->err.clear();
  }
  Outputs o{out->depth, out->id, out->normal, out->rgb, out->ao};
  ShadeParams sh = make_shade(c, s);
  cudaError_t e = run_frame_pipeline(g, sh, sc, scratch_of(c), o, sh.ssao_n > 0, c->stream, ev);
  if (e != cudaSuccess) return cuda_fail(c, e, "render_frame launch");
  return VTX_OK;
}

}  // extern "C"

// ------------------------------------------------------------ autotuner --
// Tile shape x direct-splat threshold, chosen by timing every candidate on
// the caller's own frame (or first frames of a batch) once per problem class.
static const int kTuneShapes[3][2] = {{16, 16}, {32, 8}, {8, 8}};
static const int kTuneSplat[3] = {4, 16, 64};

static int ilog2ll(long long v) {
  int r = 0;
  while (v > 1) {
    v >>= 1;
    ++r;
  }
  return r;
}

// fn(settings) enqueues one run; returns the milliseconds it took (after a sync), or < 0 on error.
template <class Fn>
static vtx_status tune(vtx_ctx *c, const long long key[6], const vtx_settings *s, vtx_settings *chosen, Fn run) {
  *chosen = *s;
  for (auto &t : c->tunes)
    if (std::equal(t.key, t.key + 6, key)) {
      chosen->tile_w = t.tw;
      chosen->tile_h = t.th;
      chosen->splat_max_px = t.splat;
      c->last_tw = t.tw;
      c->last_th = t.th;
      c->last_splat = t.splat;
      return VTX_OK;
    }
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  float best = 3.4e38f;
  int bi = 0, bj = 1;
  vtx_status st = VTX_OK;
  for (int i = 0; i < 3 && !st; ++i)
    for (int j = 0; j < 3 && !st; ++j) {
      vtx_settings cand = *s;
      cand.tile_w = kTuneShapes[i][0];
      cand.tile_h = kTuneShapes[i][1];
      cand.splat_max_px = kTuneSplat[j];
      cand.flags &= ~(uint32_t)(VTX_FLAG_SYNC | VTX_FLAG_PROFILE | VTX_FLAG_PROFILE_CULL);
      // warm-up (also grows the arena), then one timed run
      for (int attempt = 0; attempt < 4; ++attempt) {
        st = run(&cand);
        if (st) break;
        st = check_status(c);
        if (st != VTX_ERR_CAPACITY) break;
        c->err.clear();
        st = VTX_OK;
      }
      if (st) break;
      cudaEventRecord(e0, c->stream);
      st = run(&cand);
      cudaEventRecord(e1, c->stream);
      if (st) break;
      cudaEventSynchronize(e1);
      float ms = 0.0f;
      cudaEventElapsedTime(&ms, e0, e1);
      if (ms < best) {
        best = ms;
        bi = i;
        bj = j;
      }
    }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st) return st;
  vtx_ctx::Tune t;
  std::copy(key, key + 6, t.key);
  t.tw = kTuneShapes[bi][0];
  t.th = kTuneShapes[bi][1];
  t.splat = kTuneSplat[bj];
  c->tunes.push_back(t);
  chosen->tile_w = t.tw;
  chosen->tile_h = t.th;
  chosen->splat_max_px = t.splat;
  c->last_tw = t.tw;
  c->last_th = t.th;
  c->last_splat = t.splat;
  return VTX_OK;
}

extern "C" {

vtx_status vtx_render_frame(vtx_ctx *c, const vtx_settings *s, const vtx_outputs *out) {
  if (!c) return VTX_ERR_INVALID_ARG;
  cudaSetDevice(c->device);
  vtx_status st = settings_ok(c, s);
  if (st) return st;
  if (!out || !out->depth || !out->id || !out->normal || !out->rgb)
    return fail(c, VTX_ERR_INVALID_ARG, "outputs: depth, id, normal and rgb are required");
  if (!c->has_cam) return fail(c, VTX_ERR_STATE, "no camera set");
  if (c->n_atoms > 0 && !c->xyzr) return fail(c, VTX_ERR_STATE, "no atoms uploaded");
  if ((s->mode == VTX_MODE_BALL_AND_STICK || s->mode == VTX_MODE_STICKS) && c->n_bonds > 0 && c->n_atoms == 0)
    return fail(c, VTX_ERR_STATE, "bonds without atoms");
  vtx_outputs od;
  if ((st = visible_outputs(c, out, &od))) return st;
  out = &od;
  vtx_settings tuned;
  if (s->tile_w == 0) {
    const long long key[6] = {0, c->cam.width, c->cam.height, 1, ilog2ll(c->n_atoms + c->n_bonds + 1), s->mode};
    st = tune(c, key, s, &tuned, [&](const vtx_settings *cand) { return render_once(c, cand, out, nullptr); });
    if (st) return st;
    s = &tuned;
  }
  for (int attempt = 0; attempt < 4; ++attempt) {
    StageEvents ev;
    st = render_once(c, s, out, events_for(c, s, ev));
    if (st) return st;
    if (!(s->flags & VTX_FLAG_SYNC)) return VTX_OK;
    st = check_status(c);
    if (st != VTX_ERR_CAPACITY) return st;
    c->err.clear();
  }
  return st;
}

vtx_status vtx_render_frame_host(vtx_ctx *c, const float *xyzr_host, const uint8_t *elem_host,
                                 const float *palette_rgb, int32_t n_elem, int64_t n_atoms, const vtx_camera *cam,
                                 const vtx_settings *s, const vtx_outputs *oh) {
  if (!c) return VTX_ERR_INVALID_ARG;
  cudaSetDevice(c->device);
  if (n_atoms < 0 || (n_atoms > 0 && !xyzr_host) || !oh || !oh->depth || !oh->id || !oh->normal || !oh->rgb)
    return fail(c, VTX_ERR_INVALID_ARG, "host render: bad pointers");
  vtx_status st;
  if ((st = ensure(c, c->hostin_x, sizeof(float4) * (size_t)(n_atoms > 0 ? n_atoms : 1), "host atoms"))) return st;
  if (elem_host && (st = ensure(c, c->hostin_e, (size_t)(n_atoms > 0 ? n_atoms : 1), "host elements"))) return st;
  cudaError_t e = cudaMemcpyAsync(c->hostin_x.p, xyzr_host, sizeof(float4) * (size_t)n_atoms,
                                  cudaMemcpyHostToDevice, c->stream);
  if (e == cudaSuccess && elem_host)
    e = cudaMemcpyAsync(c->hostin_e.p, elem_host, (size_t)n_atoms, cudaMemcpyHostToDevice, c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "host render upload");
  if ((st = vtx_upload_atoms(c, (const float *)c->hostin_x.p, elem_host ? (const uint8_t *)c->hostin_e.p : nullptr,
                             palette_rgb, n_elem, n_atoms)))
    return st;
  if ((st = vtx_set_camera(c, cam))) return st;
  const long long ppi = (long long)cam->width * cam->height;
  size_t need = sizeof(float) * (size_t)ppi * 9;
  if ((st = ensure(c, c->hostout, need, "host outputs"))) return st;
  float *base = (float *)c->hostout.p;
  vtx_outputs od{base, (uint32_t *)(base + ppi), base + 2 * ppi, base + 5 * ppi, oh->ao ? base + 8 * ppi : nullptr};
  vtx_settings s2 = *s;
  s2.flags &= ~VTX_FLAG_SYNC;
  if ((st = vtx_render_frame(c, &s2, &od))) return st;
  e = cudaMemcpyAsync(oh->depth, od.depth, sizeof(float) * ppi, cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(oh->id, od.id, sizeof(uint32_t) * ppi, cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(oh->normal, od.normal, sizeof(float) * 3 * ppi, cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(oh->rgb, od.rgb, sizeof(float) * 3 * ppi, cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess && oh->ao)
    e = cudaMemcpyAsync(oh->ao, od.ao, sizeof(float) * ppi, cudaMemcpyDeviceToHost, c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "host render download");
  return check_status(c);
}

static vtx_status batch_once(vtx_ctx *c, const float *frames, int64_t stride, const long long *d_counts,
                             int32_t f0, int32_t nf, const vtx_camera *cams, int32_t n_views, const vtx_settings *s,
                             const vtx_outputs *out, StageEvents *ev) {
  Geometry g;
  int tw = s->tile_w ? s->tile_w : 16, th = s->tile_h ? s->tile_h : 16;
  base_geometry(g, cams, n_views, tw, th);
  g.n_frames = nf;
  g.n_img = nf * n_views;
  set_representation(g, s);
  g.splat_max = s->splat_max_px ? s->splat_max_px : default_splat(stride, g.pix_per_img);
  g.stride = stride;
  g.n_atoms = stride;
  // room for the holes the batch cull's per-warp slabs may leave (up to 4 views)
  g.surv_cap = n_views <= 4 ? stride + cull_multi_slack(stride, nf) : stride;
  g.occl = 1;  // trajectory frames of a whole system: the occlusion pass where survivors crowd the pixels
  vtx_status st = prepare(c, g, false, 0);
  if (st) return st;
  const long long ppi = g.pix_per_img;
  const long long img0 = (long long)f0 * n_views;
  g.dbg_first_wait = c->dbg_first_wait;
  Scene sc{(const float4 *)frames + (long long)f0 * stride, d_counts + f0, c->elem, nullptr, nullptr};
  sc.dbg_corrupt_key = c->dbg_corrupt_key;
  Outputs o{out->depth + img0 * ppi, out->id + img0 * ppi, out->normal + img0 * 3 * ppi, out->rgb + img0 * 3 * ppi,
            out->ao ? out->ao + img0 * ppi : nullptr};
  ShadeParams sh = make_shade(c, s);
  cudaError_t e = run_frame_pipeline(g, sh, sc, scratch_of(c), o, sh.ssao_n > 0, c->stream, ev);
  if (e != cudaSuccess) return cuda_fail(c, e, "render_batch launch");
  return VTX_OK;
}

// Frames per pipeline pass: bounded so the per-image scratch (keys and coverage list per pixel; survivor and
// kept-survivor slots per atom) stays near 8 GB, and the images of a pass within the 65,535
// blocks of a launch's second grid dimension.
static int batch_chunk(const vtx_camera *cams, int n_views, long long stride, int n_frames) {
  double per_frame = (double)n_views * ((double)cams[0].width * cams[0].height * 12.0 + (double)stride * 8.0);
  int fc = (int)(8e9 / (per_frame > 1.0 ? per_frame : 1.0));
  if (fc > 65535 / n_views) fc = 65535 / n_views;
  if (fc < 1) fc = 1;
  if (fc > n_frames) fc = n_frames;
  return fc;
}

static vtx_status batch_all(vtx_ctx *c, const float *frames, int64_t stride, const long long *d_counts, int32_t nf,
                            const vtx_camera *cams, int32_t n_views, const vtx_settings *s, const vtx_outputs *out,
                            StageEvents *ev) {
  const int fc = batch_chunk(cams, n_views, stride, nf);
  for (int f0 = 0; f0 < nf; f0 += fc) {
    int n = nf - f0 < fc ? nf - f0 : fc;
    vtx_status st = batch_once(c, frames, stride, d_counts, f0, n, cams, n_views, s, out, f0 == 0 ? ev : nullptr);
    if (st) return st;
  }
  return VTX_OK;
}

vtx_status vtx_render_batch(vtx_ctx *c, const float *frames_xyzr, int64_t frame_stride, const int64_t *atom_counts,
                            int32_t n_frames, const vtx_camera *cams, int32_t n_views, const vtx_settings *s,
                            const vtx_outputs *out, int32_t use_graph) {
  if (!c) return VTX_ERR_INVALID_ARG;
  cudaSetDevice(c->device);
  vtx_status st = settings_ok(c, s);
  if (st) return st;
  if (s->mode != VTX_MODE_VDW && s->mode != VTX_MODE_SAS)
    return fail(c, VTX_ERR_INVALID_ARG, "batch: van der Waals or SAS mode only (no bonds)");
  if (!frames_xyzr || ((uintptr_t)frames_xyzr & 15u)) return fail(c, VTX_ERR_INVALID_ARG, "frames: NULL or unaligned");
  {
    const void *df_ = nullptr;
    if (!device_visible(c, frames_xyzr, &df_, "frames: not device memory or page-locked host memory"))
      return VTX_ERR_INVALID_ARG;
    if (((uintptr_t)df_ & 15u) != 0) return fail(c, VTX_ERR_INVALID_ARG, "frames alias must be 16-byte aligned");
    frames_xyzr = (const float *)df_;
  }
  if (n_frames < 1 || n_views < 1 || n_views > VTX_MAX_VIEWS || !cams || !atom_counts)
    return fail(c, VTX_ERR_INVALID_ARG, "batch: bad frame/view counts");
  if (frame_stride < 1 || frame_stride > 2147483647LL) return fail(c, VTX_ERR_INVALID_ARG, "frame_stride");
  for (int v = 0; v < n_views; ++v) {
    if (!cam_ok(cams + v)) return fail(c, VTX_ERR_INVALID_ARG, "invalid camera");
    if (cams[v].width != cams[0].width || cams[v].height != cams[0].height)
      return fail(c, VTX_ERR_INVALID_ARG, "batch cameras must share one size");
  }
  for (int f = 0; f < n_frames; ++f)
    if (atom_counts[f] < 0 || atom_counts[f] > frame_stride) return fail(c, VTX_ERR_INVALID_ARG, "atom_counts");
  if (!out || !out->depth || !out->id || !out->normal || !out->rgb)
    return fail(c, VTX_ERR_INVALID_ARG, "outputs: depth, id, normal and rgb are required");
  // graph cache lookup
  std::vector<unsigned char> key;
  auto push = [&key](const void *p, size_t n) {
    const unsigned char *b = (const unsigned char *)p;
    key.insert(key.end(), b, b + n);
  };
  if (use_graph) {
    push(&frames_xyzr, sizeof(void *));
    push(&frame_stride, sizeof(frame_stride));
    push(&n_frames, sizeof(n_frames));
    push(atom_counts, sizeof(int64_t) * (size_t)n_frames);
    push(cams, sizeof(vtx_camera) * (size_t)n_views);
    push(s, sizeof(vtx_settings));
    push(out, sizeof(vtx_outputs));
    push(&c->elem, sizeof(void *));
    for (auto &ge : c->graphs)
      if (ge.key == key) {
        ++c->arena_gen;
        cudaError_t e = cudaGraphLaunch(ge.exec, c->stream);
        if (e != cudaSuccess) return cuda_fail(c, e, "cudaGraphLaunch");
        return VTX_OK;
      }
  }
  // per-frame atom counts on the device
  if (n_frames > c->h_counts_cap) {
    if (c->h_counts) {
      cudaEventSynchronize(c->counts_done);
      cudaFreeHost(c->h_counts);
    }
    c->h_counts = nullptr;
    if (cudaMallocHost((void **)&c->h_counts, sizeof(long long) * (size_t)n_frames) != cudaSuccess) {
      cudaGetLastError();
      c->h_counts_cap = 0;
      return fail(c, VTX_ERR_OOM, "pinned counts");
    }
    c->h_counts_cap = n_frames;
  }
  cudaEventSynchronize(c->counts_done);
  for (int f = 0; f < n_frames; ++f) c->h_counts[f] = atom_counts[f];
  if ((st = ensure(c, c->counts, sizeof(long long) * (size_t)n_frames, "counts"))) return st;
  cudaError_t e =
      cudaMemcpyAsync(c->counts.p, c->h_counts, sizeof(long long) * (size_t)n_frames, cudaMemcpyHostToDevice, c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "counts upload");
  cudaEventRecord(c->counts_done, c->stream);
  const long long *d_counts = (const long long *)c->counts.p;
  vtx_settings tuned;
  if (s->tile_w == 0) {  // tune on the first (up to) four frames
    const long long key[6] = {1, cams[0].width, cams[0].height, n_views, ilog2ll(frame_stride + 1), s->mode};
    const int nf = n_frames < 4 ? n_frames : 4;
    st = tune(c, key, s, &tuned, [&](const vtx_settings *cand) {
      return batch_all(c, frames_xyzr, frame_stride, d_counts, nf, cams, n_views, cand, out, nullptr);
    });
    if (st) return st;
    s = &tuned;
  }
  if (!use_graph) {
    for (int attempt = 0; attempt < 4; ++attempt) {
      StageEvents ev;
      st = batch_all(c, frames_xyzr, frame_stride, d_counts, n_frames, cams, n_views, s, out, events_for(c, s, ev));
      if (st) return st;
      if (!(s->flags & VTX_FLAG_SYNC)) return VTX_OK;
      st = check_status(c);
      if (st != VTX_ERR_CAPACITY) return st;
      c->err.clear();
    }
    return st;
  }
  // first use: size the arena with a synchronous run, then capture
  for (int attempt = 0; attempt < 4; ++attempt) {
    st = batch_all(c, frames_xyzr, frame_stride, d_counts, n_frames, cams, n_views, s, out, nullptr);
    if (st) return st;
    st = check_status(c);
    if (st != VTX_ERR_CAPACITY) break;
    c->err.clear();
  }
  if (st) return st;
  GraphEntry ge;
  ge.key = key;
  if (cudaMalloc((void **)&ge.d_counts, sizeof(long long) * (size_t)n_frames) != cudaSuccess) {
    cudaGetLastError();
    return fail(c, VTX_ERR_OOM, "graph counts");
  }
  cudaMemcpyAsync(ge.d_counts, d_counts, sizeof(long long) * (size_t)n_frames, cudaMemcpyDeviceToDevice, c->stream);
  cudaStreamSynchronize(c->stream);
  cudaStream_t cap = c->stream;
  bool own = false;
  if (cap == nullptr) {  // the legacy default stream cannot be captured
    cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking);
    own = true;
  }
  e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) {
    if (own) cudaStreamDestroy(cap);
    cudaFree(ge.d_counts);
    return cuda_fail(c, e, "cudaStreamBeginCapture");
  }
  cudaStream_t saved = c->stream;
  c->stream = cap;
  st = batch_all(c, frames_xyzr, frame_stride, ge.d_counts, n_frames, cams, n_views, s, out, nullptr);
  c->stream = saved;
  cudaGraph_t graph = nullptr;
  cudaError_t e2 = cudaStreamEndCapture(cap, &graph);
  if (own) cudaStreamDestroy(cap);
  if (st || e2 != cudaSuccess) {
    if (graph) cudaGraphDestroy(graph);
    cudaFree(ge.d_counts);
    return st ? st : cuda_fail(c, e2, "cudaStreamEndCapture");
  }
  e = cudaGraphInstantiate(&ge.exec, graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) {
    cudaFree(ge.d_counts);
    return cuda_fail(c, e, "cudaGraphInstantiate");
  }
  c->graphs.push_back(ge);
  ++c->arena_gen;
  e = cudaGraphLaunch(ge.exec, c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "cudaGraphLaunch");
  return VTX_OK;
}

static vtx_status soft_common(vtx_ctx *c, const float *xyzr, int64_t n, const vtx_camera *cams, int32_t n_views,
                              float sigma, Geometry &g) {
  if (!xyzr || ((uintptr_t)xyzr & 15u)) return fail(c, VTX_ERR_INVALID_ARG, "xyzr: NULL or unaligned");
  if (n < 1 || n > 2147483647LL) return fail(c, VTX_ERR_INVALID_ARG, "n out of range");
  if (!cams || n_views < 1 || n_views > VTX_MAX_VIEWS) return fail(c, VTX_ERR_INVALID_ARG, "views");
  if (!(sigma > 0.0f)) return fail(c, VTX_ERR_INVALID_ARG, "sigma_px must be > 0");
  for (int v = 0; v < n_views; ++v) {
    if (!cam_ok(cams + v)) return fail(c, VTX_ERR_INVALID_ARG, "invalid camera");
    if (cams[v].width != cams[0].width || cams[v].height != cams[0].height)
      return fail(c, VTX_ERR_INVALID_ARG, "soft cameras must share one size");
  }
  base_geometry(g, cams, n_views, 16, 16);
  g.n_frames = 1;
  g.n_img = n_views;
  g.mode = VTX_MODE_VDW;
  g.soft = 1;
  g.sigma = sigma;
  g.stride = n;
  g.n_atoms = n;
  g.surv_cap = n;
  g.dbg_first_wait = c->dbg_first_wait;
  return prepare(c, g, true, n);
}

// Soft calls: with VTX_FLAG_SYNC (and always for the first call of a problem size on a context) the call
// synchronises, grows the arena on a capacity overflow and renders again; otherwise it only enqueues and a
// device-side error is reported by the next synchronising call.
static vtx_status soft_run(vtx_ctx *c, const float *xyzr, int64_t n, const vtx_camera *cams, int32_t n_views,
                           float sigma, uint32_t flags, float *cov, float *depth, float *normal, const float *gc,
                           const float *gd, const float *gn, float *grad, uint32_t *state) {
  if (!c) return VTX_ERR_INVALID_ARG;
  cudaSetDevice(c->device);
  if (((uintptr_t)state & 7u) != 0) return fail(c, VTX_ERR_INVALID_ARG, "state must be 8-byte aligned");
  const long long key[4] = {(long long)n, n_views, n_views >= 1 && cams ? cams[0].width : 0,
                            n_views >= 1 && cams ? cams[0].height : 0};
  const bool sized = std::equal(key, key + 4, c->soft_sized);
  const bool sync = (flags & VTX_FLAG_SYNC) != 0 || !sized;
  // a backward call may reuse the lists of the latest forward call when nothing has used the arena since and
  // the inputs are the same (the caller vouches, with the flag, that the contents of xyzr are unchanged)
  const auto &L = c->soft_lists;
  bool reuse = grad != nullptr && (flags & VTX_FLAG_SOFT_REUSE) != 0 && L.gen == c->arena_gen && L.xyzr == xyzr &&
               L.n == n && L.sigma == sigma && cams && n_views >= 1 && L.cams.size() == (size_t)n_views &&
               std::memcmp(L.cams.data(), cams, sizeof(vtx_camera) * (size_t)n_views) == 0;
  vtx_status st = VTX_OK;
  for (int attempt = 0; attempt < 4; ++attempt) {
    Geometry g;
    const uint64_t gen0 = c->arena_gen, alloc0 = c->alloc_gen;
    st = soft_common(c, xyzr, n, cams, n_views, sigma, g);
    if (st) return st;
    if (reuse && c->alloc_gen == alloc0)
      c->arena_gen = gen0;  // sizing an arena that already fits the lists leaves them in place
    else
      reuse = false;
    Scene sc{(const float4 *)xyzr, nullptr, nullptr, nullptr, nullptr};
    cudaError_t e = run_soft_pipeline(g, sc, scratch_of(c), cov, depth, normal, gc, gd, gn, grad, (uint2 *)state,
                                      reuse, c->stream, nullptr);
    if (e != cudaSuccess) return cuda_fail(c, e, "soft launch");
    if (grad == nullptr) {
      c->soft_lists.gen = c->arena_gen;
      c->soft_lists.xyzr = xyzr;
      c->soft_lists.n = n;
      c->soft_lists.sigma = sigma;
      c->soft_lists.cams.assign(cams, cams + n_views);
    }
    reuse = false;  // a retry after an overflow rebuilds everything
    if (!sync) return VTX_OK;
    st = check_status(c);
    if (st == VTX_OK) std::copy(key, key + 4, c->soft_sized);
    if (st != VTX_ERR_CAPACITY) return st;
    c->err.clear();
  }
  return st;
}

vtx_status vtx_render_soft_fwd_ex(vtx_ctx *c, const float *xyzr, int64_t n, const vtx_camera *cams,
                                  int32_t n_views, float sigma_px, uint32_t flags, float *cov, float *depth,
                                  float *normal, uint32_t *state) {
  if (!cov || !depth || !normal) return fail(c, VTX_ERR_INVALID_ARG, "soft outputs are required");
  return soft_run(c, xyzr, n, cams, n_views, sigma_px, flags, cov, depth, normal, nullptr, nullptr, nullptr,
                  nullptr, state);
}

vtx_status vtx_render_soft_bwd_ex(vtx_ctx *c, const float *xyzr, int64_t n, const vtx_camera *cams,
                                  int32_t n_views, float sigma_px, uint32_t flags, const float *g_cov,
                                  const float *g_depth, const float *g_normal, const uint32_t *state,
                                  float *grad_xyzr) {
  if (!grad_xyzr || ((uintptr_t)grad_xyzr & 15u)) return fail(c, VTX_ERR_INVALID_ARG, "grad_xyzr: NULL or unaligned");
  return soft_run(c, xyzr, n, cams, n_views, sigma_px, flags, nullptr, nullptr, nullptr, g_cov, g_depth, g_normal,
                  grad_xyzr, const_cast<uint32_t *>(state));
}

vtx_status vtx_render_soft_fwd(vtx_ctx *c, const float *xyzr, int64_t n, const vtx_camera *cams, int32_t n_views,
                               float sigma_px, float *cov, float *depth, float *normal) {
  return vtx_render_soft_fwd_ex(c, xyzr, n, cams, n_views, sigma_px, VTX_FLAG_SYNC, cov, depth, normal, nullptr);
}

vtx_status vtx_render_soft_bwd(vtx_ctx *c, const float *xyzr, int64_t n, const vtx_camera *cams, int32_t n_views,
                               float sigma_px, const float *g_cov, const float *g_depth, const float *g_normal,
                               float *grad_xyzr) {
  return vtx_render_soft_bwd_ex(c, xyzr, n, cams, n_views, sigma_px, VTX_FLAG_SYNC, g_cov, g_depth, g_normal,
                                nullptr, grad_xyzr);
}

vtx_status vtx_soft_terms(vtx_ctx *c, uint64_t *n_terms) {
  if (!c || !n_terms) return VTX_ERR_INVALID_ARG;
  cudaSetDevice(c->device);
  if (!c->status.p) {
    *n_terms = 0;
    return VTX_OK;
  }
  cudaError_t e = cudaMemcpyAsync(c->h_status, c->status.p, sizeof(Status), cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "soft terms");
  *n_terms = (uint64_t)c->h_status->n_terms;
  return VTX_OK;
}

vtx_status vtx_sync_status(vtx_ctx *c) {
  if (!c) return VTX_ERR_INVALID_ARG;
  cudaSetDevice(c->device);
  if (!c->status.p) {
    cudaError_t e = cudaStreamSynchronize(c->stream);
    return e == cudaSuccess ? VTX_OK : cuda_fail(c, e, "device error");
  }
  return check_status(c);
}

vtx_status vtx_stage_times(vtx_ctx *c, const char **names, float *ms, int32_t *n, int32_t *runs) {
  if (!c || !n) return VTX_ERR_INVALID_ARG;
  if (c->ev_used == 0) {
    *n = 0;
    if (runs) *runs = 0;
    return fail(c, VTX_ERR_STATE, "no profiled render since the last read");
  }
  const size_t last = c->ev_used - 1;
  cudaError_t e = cudaEventSynchronize(c->ev_sets[last][c->ev_masks[last] == ~0u ? kNumStages - 1 : 1]);
  if (e != cudaSuccess) return cuda_fail(c, e, "stage events");
  int cap = *n < kNumStages ? *n : kNumStages;
  double acc[kNumStages] = {};
  int cnt[kNumStages] = {};
  for (size_t r = 0; r < c->ev_used; ++r) {
    cudaEvent_t *set = c->ev_sets[r];
    if (c->ev_masks[r] != ~0u) {  // cull only
      float t = 0.0f;
      cudaEventElapsedTime(&t, set[0], set[1]);
      acc[1] += t;
      ++cnt[1];
      continue;
    }
    cudaEvent_t prev = set[kNumStages];
    for (int i = 0; i < kNumStages; ++i) {
      float t = 0.0f;
      cudaEventElapsedTime(&t, prev, set[i]);
      acc[i] += t;
      ++cnt[i];
      prev = set[i];
    }
  }
  for (int i = 0; i < cap; ++i) {
    if (names) names[i] = kStageNames[i];
    if (ms) ms[i] = cnt[i] ? (float)(acc[i] / (double)cnt[i]) : 0.0f;
  }
  *n = cap;
  if (runs) *runs = (int32_t)c->ev_used;
  c->ev_used = 0;
  return VTX_OK;
}

vtx_status vtx_tuned_settings(const vtx_ctx *c, int32_t *tile_w, int32_t *tile_h, int32_t *splat_max_px) {
  if (!c || !tile_w || !tile_h || !splat_max_px) return VTX_ERR_INVALID_ARG;
  if (c->last_tw == 0) return VTX_ERR_STATE;
  *tile_w = c->last_tw;
  *tile_h = c->last_th;
  *splat_max_px = c->last_splat;
  return VTX_OK;
}

vtx_status vtx_export_rgba8(vtx_ctx *c, const float *rgb, const uint32_t *id, int32_t width, int32_t height,
                            int32_t n_images, float background_alpha, uint8_t *rgba) {
  if (!c) return VTX_ERR_INVALID_ARG;
  if (width < 1 || height < 1 || width > 16384 || height > 16384 || n_images < 1)
    return fail(c, VTX_ERR_INVALID_ARG, "export: bad image size or count");
  if (!rgb || !id || !rgba) return fail(c, VTX_ERR_INVALID_ARG, "export: NULL plane");
  if (((uintptr_t)rgba & 3u) != 0) return fail(c, VTX_ERR_INVALID_ARG, "export: rgba must be 4-byte aligned");
  if (!(background_alpha == background_alpha)) return fail(c, VTX_ERR_INVALID_ARG, "export: background_alpha is NaN");
  cudaSetDevice(c->device);
  const void *dr = nullptr, *di = nullptr, *dout = nullptr;
  if (!device_visible(c, rgb, &dr, "export: rgb not device or page-locked host memory") ||
      !device_visible(c, id, &di, "export: id not device or page-locked host memory") ||
      !device_visible(c, rgba, &dout, "export: rgba not device or page-locked host memory"))
    return VTX_ERR_INVALID_ARG;
  if (((uintptr_t)dout & 3u) != 0) return fail(c, VTX_ERR_INVALID_ARG, "export: rgba alias must be 4-byte aligned");
  const unsigned char bg_a = (unsigned char)std::lrint(255.0f * std::fmin(std::fmax(background_alpha, 0.0f), 1.0f));
  cudaError_t e = run_export_rgba8((const float *)dr, (const uint32_t *)di, (long long)width * height, n_images,
                                   bg_a, (uint8_t *)dout, c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "export launch");
  return VTX_OK;
}

vtx_status vtx_ses_fit_grid(vtx_ctx *c, const float *xyzr, int64_t n_atoms, float probe, float spacing,
                            vtx_ses_grid *g) {
  if (!c) return VTX_ERR_INVALID_ARG;
  if (!g || n_atoms < 1 || !xyzr) return fail(c, VTX_ERR_INVALID_ARG, "ses grid: need atoms and an output");
  if (!(spacing > 0.0f) || !(probe >= 0.0f) || !std::isfinite(spacing) || !std::isfinite(probe))
    return fail(c, VTX_ERR_INVALID_ARG, "ses grid: spacing > 0 and probe >= 0 required");
  cudaSetDevice(c->device);
  const void *dx = nullptr;
  if (!device_visible(c, xyzr, &dx, "ses: xyzr not device or page-locked host memory")) return VTX_ERR_INVALID_ARG;
  if (((uintptr_t)dx & 15u) != 0) return fail(c, VTX_ERR_INVALID_ARG, "ses: xyzr must be 16-byte aligned");
  const int nb = 4 * sm_count();
  vtx_status st = ensure(c, c->ses_bbox, sizeof(float) * 6 * (size_t)nb, "ses bbox");
  if (st) return st;
  cudaError_t e = run_ses_bbox((const float4 *)dx, n_atoms, probe, (float *)c->ses_bbox.p, nb, c->stream);
  std::vector<float> part((size_t)nb * 6);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(part.data(), c->ses_bbox.p, sizeof(float) * part.size(), cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "ses bbox");
  float lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
  for (int b = 0; b < nb; ++b)
    for (int d = 0; d < 3; ++d) {
      lo[d] = std::fmin(lo[d], part[(size_t)b * 6 + d]);
      hi[d] = std::fmax(hi[d], part[(size_t)b * 6 + 3 + d]);
    }
  for (int d = 0; d < 3; ++d) {
    if (!std::isfinite(lo[d]) || !std::isfinite(hi[d])) return fail(c, VTX_ERR_INVALID_ARG, "ses: non-finite atoms");
    g->origin[d] = (float)((double)lo[d] - 2.0 * (double)spacing);
    const double n = std::floor(((double)hi[d] - (double)lo[d]) / (double)spacing) + 6.0;
    if (n > 2147483647.0) return fail(c, VTX_ERR_INVALID_ARG, "ses: grid too large");
    g->dims[d] = (int32_t)n;
  }
  g->spacing = spacing;
  g->probe = probe;
  return VTX_OK;
}

vtx_status vtx_ses_mesh(vtx_ctx *c, const float *xyzr, int64_t n_atoms, const vtx_ses_grid *g, float *tris,
                        int64_t max_tris, int64_t *labels, uint8_t *sas, uint16_t *edt2, int64_t *n_tris) {
  if (!c) return VTX_ERR_INVALID_ARG;
  if (!g || !n_tris || max_tris < 0 || (max_tris > 0 && !tris) || n_atoms < 0 || (n_atoms > 0 && !xyzr))
    return fail(c, VTX_ERR_INVALID_ARG, "ses: bad arguments");
  if (!(g->spacing > 0.0f) || !(g->probe >= 0.0f) || !std::isfinite(g->spacing) || !std::isfinite(g->probe) ||
      (double)g->probe / (double)g->spacing > 150.0)
    return fail(c, VTX_ERR_INVALID_ARG, "ses: spacing > 0, probe >= 0 and probe / spacing <= 150 required");
  for (int d = 0; d < 3; ++d)
    if (g->dims[d] < 2 || !std::isfinite(g->origin[d])) return fail(c, VTX_ERR_INVALID_ARG, "ses: dims >= 2");
  const long long n_pts = (long long)g->dims[0] * g->dims[1] * g->dims[2];
  if (n_pts > 4294967296LL) return fail(c, VTX_ERR_INVALID_ARG, "ses: more than 2^32 grid points");
  cudaSetDevice(c->device);
  const void *dx = nullptr, *dt = nullptr, *dl = nullptr, *ds = nullptr, *de = nullptr;
  if (!device_visible(c, xyzr, &dx, "ses: xyzr not device or page-locked host memory") ||
      !device_visible(c, tris, &dt, "ses: tris not device or page-locked host memory") ||
      !device_visible(c, labels, &dl, "ses: labels not device or page-locked host memory") ||
      !device_visible(c, sas, &ds, "ses: sas not device or page-locked host memory") ||
      !device_visible(c, edt2, &de, "ses: edt2 not device or page-locked host memory"))
    return VTX_ERR_INVALID_ARG;
  if (((uintptr_t)dx & 15u) != 0) return fail(c, VTX_ERR_INVALID_ARG, "ses: xyzr must be 16-byte aligned");
  if (((uintptr_t)dt & 3u) != 0 || ((uintptr_t)dl & 7u) != 0 || ((uintptr_t)de & 1u) != 0)
    return fail(c, VTX_ERR_INVALID_ARG, "ses: misaligned output");
  const long long nb = ses_blocks(g->dims);
  vtx_status st;
  if (!ds && (st = ensure(c, c->ses_sas, (size_t)n_pts, "ses sas"))) return st;
  if ((st = ensure(c, c->ses_a, 2 * (size_t)n_pts, "ses pass a"))) return st;
  if ((st = ensure(c, c->ses_b, 2 * (size_t)n_pts, "ses pass b"))) return st;
  if (!de && (st = ensure(c, c->ses_edt, 2 * (size_t)n_pts, "ses edt"))) return st;
  if ((st = ensure(c, c->ses_blk, sizeof(unsigned) * (size_t)(nb + 1), "ses blocks"))) return st;
  if ((st = ensure(c, c->ses_case, (size_t)n_pts, "ses cases"))) return st;  // >= one byte per cell
  if ((st = ensure(c, c->ses_base, sizeof(unsigned long long) * (size_t)(nb + 1), "ses bases"))) return st;
  if ((st = ensure(c, c->ses_total, sizeof(unsigned long long), "ses total"))) return st;
  SesLaunch L;
  L.X = (const float4 *)dx;
  L.n_atoms = n_atoms;
  for (int d = 0; d < 3; ++d) {
    L.origin[d] = g->origin[d];
    L.dims[d] = g->dims[d];
  }
  L.h = g->spacing;
  L.probe = g->probe;
  L.sas = ds ? (uint8_t *)ds : (uint8_t *)c->ses_sas.p;
  L.g_a = (uint16_t *)c->ses_a.p;
  L.g_b = (uint16_t *)c->ses_b.p;
  L.edt2 = de ? (uint16_t *)de : (uint16_t *)c->ses_edt.p;
  L.cases = (uint8_t *)c->ses_case.p;
  L.block_tris = (unsigned *)c->ses_blk.p;
  L.block_base = (unsigned long long *)c->ses_base.p;
  L.total = (unsigned long long *)c->ses_total.p;
  L.tris = (float *)dt;
  L.labels = (long long *)dl;
  L.max_tris = max_tris;
  cudaError_t e = run_ses_grid(L, c->stream);
  unsigned long long total = 0;
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(&total, L.total, sizeof(total), cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "ses mesh");
  *n_tris = (int64_t)total;
  if ((long long)total > max_tris) return fail(c, VTX_ERR_CAPACITY, "ses: more triangles than max_tris");
  return VTX_OK;
}

vtx_status vtx_debug_hooks(vtx_ctx *c, int32_t first_wait_polls, uint32_t cap_records, uint64_t cap_entries,
                           int32_t corrupt_key) {
  if (!c) return VTX_ERR_INVALID_ARG;
  c->dbg_first_wait = first_wait_polls < 0 ? -1 : first_wait_polls;
  c->dbg_corrupt_key = corrupt_key != 0;
  if (cap_records > 0) c->cap_rec = cap_records;
  if (cap_entries > 0) c->cap_entries = cap_entries;
  drop_graphs(c);
  return VTX_OK;
}

const char *vtx_last_error(const vtx_ctx *c) { return c ? c->err.c_str() : "null context"; }

}  // extern "C"
