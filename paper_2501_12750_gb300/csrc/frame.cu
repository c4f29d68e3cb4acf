// frame.cu -- per-frame hard-edge path of the meshless ray-caster.
//
// The paper rasterises one impostor quad per primitive and ray-casts the
// implicit surface in a fragment shader (Methods, "Meshless
// Representations"), then shades a G-buffer and runs screen-space ambient
// occlusion ("High Quality Rendering").  Here the same per-pixel result --
// the nearest ray/primitive hit -- is computed without a graphics API:
//
//   k_clear      resets image states and counters, tile counts and (single
//        frames) keys; a batch's key planes are cleared by a byte memset;
//   k_cull_direct / k_cull_multi / k_cull_atoms / k_cull_bonds  stream every
//        record once (one view; a batch of up to four views; more views),
//        reject what cannot cover a pixel centre, append survivors through
//        per-warp slabs or per-block runs;
//   k_setup      fixes each image's depth-key range from the survivors, then
//        precise double-float setup per survivor; footprints of at
//        most splat_max candidate pixels are ray-cast right there and
//        merged with a 64-bit atomicMin of (depth key << 32 | id); larger
//        ones become 64-byte records counted per screen tile;
//   k_occl_upper / k_occl_test  (crowded batch images) the front survivors
//        write bound keys (FP32 upper bounds of their entry depth, as keys)
//        at the pixels they certainly cover; setup then takes only the
//        survivors that these keys do not hide at every pixel of their boxes;
//   k_scan_*     exclusive scan of the per-tile counts (counting sort by tile),
//        listing the non-empty tiles longest first;
//   k_scatter    writes (min depth key << 32 | record) entries per tile;
//   k_raster     resident CTAs take tiles from a queue: each orders its tile's
//        entries front to back by depth bucket in shared memory (one-pass
//        counting sort) with a pixel box per entry; then each warp walks the
//        ordered list on its own, staging 32 records at a time (only those
//        whose boxes meet its still-searching pixels), dropping those whose
//        bounding sphere misses every ray of those pixels, ray-casting the
//        rest two at a time, and stopping once every pixel's hit is nearer
//        than the next entry's nearest possible depth;
//   k_resolve_list / k_resolve_split  list the covered pixels, then shade
//        them (id decoded, hit recomputed -> depth, normal, colour, SSAO
//        from neighbouring depth keys, outline, fog) beside CTAs that write
//        the background pixels; every output plane is written once.
#include <cstdio>

#include "vtx_internal.h"

namespace vtx {

constexpr int kCullThreads = 256;
constexpr int kStages = 2;                           // TMA pipeline depth of the cull
constexpr int kChunk = 1024;                         // atoms per stage (16 KB)
constexpr int kPerThread = kChunk / kCullThreads;
constexpr size_t kCullSmem = (size_t)kStages * kChunk * sizeof(float4);
constexpr uint32_t kWaitLimit = 1u << 24;            // polls before a wait is declared failed
constexpr int kScanItems = 4096;  // tiles per scan block (1024 threads x 4)

int sm_count() {
  static int n = 0;
  if (n == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    if (n <= 0) n = 132;
  }
  return n;
}

// ----------------------------------------------------------------- init --

// Frame set-up in one launch: image states and launch counters reset, tile
// counts zeroed and (hard edges) every depth key set to the background key.
__global__ __launch_bounds__(256) void k_clear(ImageState *st, int n_img, Status *status, uint32_t *tile_count,
                                               long long n_tiles, unsigned long long *keys, long long n_keys) {
  pdl_enter();
  const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long stride = (long long)gridDim.x * blockDim.x;
  if (tid < n_img) {
    ImageState s;
    s.zlo_bits = 0x7f800000u;
    s.zhi_bits = 0u;
    s.n_surv = 0u;
    s.valid = 0u;
    s.zlo = 0.0f;
    s.S = 0.0f;
    s.invS = 0.0f;
    s.occl = 0u;
    s.n_vis = 0u;
    st[tid] = s;
  }
  if (tid == 0) {
    status->n_rec = 0u;
    status->n_entries = 0ull;
    status->n_terms = 0ull;
    status->soft_next = 0u;
    status->tile_next = 0u;
    status->n_list = 0u;
    status->n_cov = 0u;
  }
  for (long long i = tid; i < n_tiles; i += stride) tile_count[i] = 0u;
  // keys: 16-byte stores over the (256-byte aligned) buffer, then the odd tail
  const ulonglong2 bg2 = make_ulonglong2(kBgKey, kBgKey);
  ulonglong2 *k2 = reinterpret_cast<ulonglong2 *>(keys);
  for (long long i = tid; i < n_keys / 2; i += stride) k2[i] = bg2;
  if ((n_keys & 1) && tid == 0) keys[n_keys - 1] = kBgKey;
}

// ----------------------------------------------------------------- cull --

// Radius used for binning.  Soft mode dilates by 4 px at the centre depth
// (primitives contribute while their signed pixel distance is >= -4 px).
__device__ __forceinline__ float cull_radius(const Geometry &g, const ViewParams &v, float r, float z) {
  if (g.soft) return r + 4.0f * fmaxf(z, 0.0f) * v.inv_f * 1.0001f + 1e-6f;
  return r;
}

__device__ __forceinline__ void warp_minmax(float &lo, float &hi) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    lo = fminf(lo, __shfl_xor_sync(0xffffffffu, lo, o));
    hi = fmaxf(hi, __shfl_xor_sync(0xffffffffu, hi, o));
  }
}

// Every atom record of frame blockIdx.y is read once and tested against all
// views of that frame.  The records stream through shared memory in
// kStages x 16 KB stages filled by 1-D TMA bulk copies (cp.async.bulk,
// completion on an mbarrier), so HBM reads overlap the tests of earlier
// stages.  Survivors are compacted per view with warp ballots into shared
// memory and appended with one global atomic per 1,024 atoms.
// ONE_VIEW: a single camera, whose constants are then compile-time indexed
// kernel parameters; otherwise the views are read from a shared-memory copy.
// blockIdx.z splits the views into gridDim.z groups (each CTA tests its
// group only): a few atoms seen from many views then still fill the GPU.
template <bool ONE_VIEW>
__global__ __launch_bounds__(kCullThreads, 5) void k_cull_atoms(Geometry g, const float4 *__restrict__ frames,
                                                                const long long *__restrict__ counts, ImageState *st,
                                                                uint32_t *__restrict__ surv, Status *status) {
  pdl_enter();
  extern __shared__ __align__(128) unsigned char cull_smem[];
  float4 *s_atoms = reinterpret_cast<float4 *>(cull_smem);
  __shared__ ViewParams s_views[ONE_VIEW ? 1 : kMaxViews];
  __shared__ __align__(8) uint64_t s_bar[kStages];
  __shared__ uint32_t s_idx[3][kChunk];
  __shared__ int s_cnt[3];
  __shared__ unsigned int s_pub_base;
  __shared__ int s_pub_cnt, s_pub_img;
  __shared__ int s_fail;
  __shared__ unsigned int s_zlo[kMaxViews], s_zhi[kMaxViews];
  const int frame = blockIdx.y;
  const long long n = counts ? counts[frame] : g.n_atoms;
  const float4 *X = frames + (long long)frame * g.stride;
  const long long n_chunks = (n + kChunk - 1) / kChunk;
  const long long mine = (long long)blockIdx.x < n_chunks ? (n_chunks - 1 - blockIdx.x) / gridDim.x + 1 : 0;
  const int lane = threadIdx.x & 31;
  if (threadIdx.x < kMaxViews) {
    s_zlo[threadIdx.x] = 0x7f800000u;
    s_zhi[threadIdx.x] = 0u;
    if (!ONE_VIEW && threadIdx.x < g.n_views) s_views[threadIdx.x] = g.views[threadIdx.x];
  }
  const int vper = ONE_VIEW ? 1 : (g.n_views + (int)gridDim.z - 1) / (int)gridDim.z;
  const int v_begin = ONE_VIEW ? 0 : min((int)blockIdx.z * vper, g.n_views);
  const int v_end = ONE_VIEW ? 1 : min(v_begin + vper, g.n_views);
  if (threadIdx.x == 0) {
    s_fail = 0;
    s_cnt[0] = 0;
    s_cnt[1] = 0;
    s_cnt[2] = 0;
    for (int s = 0; s < kStages; ++s) mbar_init(&s_bar[s], 1u);
    fence_mbar_init();
  }
  __syncthreads();
  long long issued = 0;  // meaningful in thread 0 only
  if (threadIdx.x == 0) {
    for (; issued < mine && issued < kStages; ++issued) {
      const long long a0 = ((long long)blockIdx.x + issued * gridDim.x) * kChunk;
      const uint32_t bytes = (uint32_t)min((long long)kChunk, n - a0) * 16u;
      const int stg = (int)(issued % kStages);
      mbar_expect_tx(&s_bar[stg], bytes);
      bulk_g2s(s_atoms + stg * kChunk, X + a0, bytes, &s_bar[stg]);
    }
  }
  // Survivors of unit u = (chunk, view) collect in s_idx[u % 3]; the global
  // atomic that reserves their slots is issued at unit u and its result is
  // consumed one unit later, so its latency hides behind the next unit.
  int ub = 0;  // buffer of the current unit: u % 3
  int stg = 0;
  uint32_t phase = 0u;
  unsigned int pend_base = 0u;  // thread 0: atomic result of the previous unit
  int pend_cnt = 0, pend_img = 0;
  long long k = 0;
  for (; k < mine; ++k) {
    // stage k % kStages, parity (k / kStages) & 1
    // the normal poll limit, except for a test hook that shortens the first wait (the drain below keeps it)
    const uint32_t lim = (k == 0 && g.dbg_first_wait >= 0) ? (uint32_t)g.dbg_first_wait : kWaitLimit;
    if (!mbar_wait_bounded(&s_bar[stg], phase, lim)) {
      s_fail = 1;
      atomicOr(&status->overflow, 16u);
    }
    const long long a0 = ((long long)blockIdx.x + k * gridDim.x) * kChunk;
    const int cnt = (int)min((long long)kChunk, n - a0);
    float4 a[kPerThread];
#pragma unroll
    for (int j = 0; j < kPerThread; ++j) {
      const int i = j * kCullThreads + threadIdx.x;
      a[j] = i < cnt ? s_atoms[stg * kChunk + i] : make_float4(0.0f, 0.0f, 0.0f, -1.0f);
    }
    for (int v = v_begin; v < v_end; ++v, ub = ub == 2 ? 0 : ub + 1) {
      const int b = ub;
      const ViewParams &vp = ONE_VIEW ? g.views[0] : s_views[v];
      float zlo = __int_as_float(0x7f800000), zhi = 0.0f;
#pragma unroll
      for (int j = 0; j < kPerThread; ++j) {
        bool keep = false;
        if (a[j].w >= 0.0f) {
          const float r = atom_radius(g, a[j].w);
          float vx, vy, vz, err;
          view_f32(vp, a[j].x, a[j].y, a[j].z, vx, vy, vz, err);
          const float R = cull_radius(g, vp, r, vz);
          keep = cull_lean(vp, vx, vy, vz, R + err) && clip_keep(g, a[j].x, a[j].y, a[j].z);
          if (g.soft && !(vz > vp.znear)) keep = false;
          if (keep) {
            zlo = fminf(zlo, vz - R - err);
            zhi = fmaxf(zhi, vz + R + err);
          }
        }
        const unsigned m = __ballot_sync(0xffffffffu, keep);
        if (m) {
          const int leader = __ffs(m) - 1;
          int pos = 0;
          if (lane == leader) pos = atomicAdd(&s_cnt[b], __popc(m));
          pos = __shfl_sync(0xffffffffu, pos, leader);
          if (keep) s_idx[b][pos + __popc(m & ((1u << lane) - 1u))] = (uint32_t)(a0 + j * kCullThreads + threadIdx.x);
        }
      }
      warp_minmax(zlo, zhi);
      if (lane == 0 && zhi > 0.0f) {
        atomicMin(&s_zlo[v], __float_as_uint(fmaxf(zlo, 0.0f)));
        atomicMax(&s_zhi[v], __float_as_uint(zhi));
      }
      __syncthreads();  // (A) unit u collected; every thread holds its atoms in registers
      if (threadIdx.x == 0) {
        // publish the previous unit's reservation (its atomic has long returned)
        s_pub_base = pend_base;
        s_pub_cnt = pend_cnt;
        s_pub_img = pend_img;
        // reserve this unit's slots; the result is only read at the next unit
        const int img = frame * g.n_views + v;
        const int c = s_cnt[b];
        pend_base = c ? atomicAdd(&st[img].n_surv, (unsigned)c) : 0u;
        pend_cnt = c;
        pend_img = img;
        s_cnt[(b + 1) % 3] = 0;
        if (v == v_begin && issued < mine) {  // the stage is free again: refill it
          fence_proxy_async();
          const long long b0 = ((long long)blockIdx.x + issued * gridDim.x) * kChunk;
          const uint32_t bytes = (uint32_t)min((long long)kChunk, n - b0) * 16u;
          const int s2 = (int)(issued % kStages);
          mbar_expect_tx(&s_bar[s2], bytes);
          bulk_g2s(s_atoms + s2 * kChunk, X + b0, bytes, &s_bar[s2]);
          ++issued;
        }
      }
      __syncthreads();  // (B)
      {  // write out the previous unit
        const int c = s_pub_cnt;
        const int pb = b == 0 ? 2 : b - 1;
        uint32_t *dst = surv + (long long)s_pub_img * g.surv_cap + s_pub_base;
        for (int i = threadIdx.x; i < c; i += kCullThreads) dst[i] = s_idx[pb][i];
      }
    }
    if (++stg == kStages) {
      stg = 0;
      phase ^= 1u;
    }
    if (s_fail) break;  // uniform: s_fail is only written before barrier (A) of a chunk
  }
  // the last unit's survivors
  __syncthreads();
  if (threadIdx.x == 0) {
    s_pub_base = pend_base;
    s_pub_cnt = pend_cnt;
    s_pub_img = pend_img;
  }
  __syncthreads();
  {
    const int c = s_pub_cnt;
    const int pb = ub == 0 ? 2 : ub - 1;
    uint32_t *dst = surv + (long long)s_pub_img * g.surv_cap + s_pub_base;
    for (int i = threadIdx.x; i < c; i += kCullThreads) dst[i] = s_idx[pb][i];
  }
  // drain copies still in flight (only after a failed wait)
  if (threadIdx.x == 0) {
    for (long long q = k; q < issued; ++q)
      mbar_wait_bounded(&s_bar[q % kStages], (uint32_t)((q / kStages) & 1), kWaitLimit);
  }
  __syncthreads();
  if ((int)threadIdx.x >= v_begin && (int)threadIdx.x < v_end && s_zhi[threadIdx.x] != 0u) {
    const int img = frame * g.n_views + threadIdx.x;
    atomicMin(&st[img].zlo_bits, s_zlo[threadIdx.x]);
    atomicMax(&st[img].zhi_bits, s_zhi[threadIdx.x]);
  }
}

// Survivor slab size: one global atomic per slab.  On the close view (tens of
// millions of survivors) the shared counter was the cull's bottleneck at 64
// slots (0.84 ms; 128: 0.61 ms; 256: 0.30 ms); at 1024 the holes (a warp's
// last slab) start to cost setup time on the overview.
#ifndef VTX_SLAB
#define VTX_SLAB 256
#endif
constexpr int kSlab = VTX_SLAB;  // survivor slots a warp reserves at a time (single-view cull)

// Warp-aggregated survivor append through per-warp slabs: slots [used, kSlab)
// of the current slab first, the rest in a fresh slab reserved with one
// global atomic.  All 32 lanes call it together.
__device__ __forceinline__ void slab_push(bool keep, uint32_t idx, int lane, unsigned lt, uint32_t &slab, int &used,
                                          unsigned *n_surv, uint32_t *__restrict__ surv, long long cap) {
  const unsigned m = __ballot_sync(0xffffffffu, keep);
  if (!m) return;
  const int c = __popc(m);
  const int pos = used + __popc(m & lt);
  uint32_t next = slab;
  if (used + c > kSlab) {
    unsigned nb = 0u;
    if (lane == 0) nb = atomicAdd(n_surv, (unsigned)kSlab);
    next = __shfl_sync(0xffffffffu, nb, 0);
  }
  if (keep) {
    const long long dst = pos < kSlab ? (long long)slab + pos : (long long)next + (pos - kSlab);
    if (dst < cap) surv[dst] = idx;
  }
  if (used + c > kSlab) {
    slab = next;
    used = used + c - kSlab;
  } else {
    used += c;
  }
}

// Setup CTAs per image in batches of 64 or more images (16: measured against 4 and 8).
#ifndef VTX_SETUP_BATCH_CTAS
#define VTX_SETUP_BATCH_CTAS 16
#endif
// The cull's streaming load: read-only, not kept in L1, 256-byte L2 requests
// (measured 1 % ahead of an evict-first load and 4 % ahead of a plain __ldg).
__device__ __forceinline__ float4 cull_load(const float4 *p) {
  float4 v;
  asm volatile("ld.global.nc.L1::no_allocate.L2::256B.v4.f32 {%0, %1, %2, %3}, [%4];"
               : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
               : "l"(p));
  return v;
}
constexpr int kCullPT = 4;          // atoms per thread per pass of the single-view cull
constexpr int kCullCtasPerSm = 5;   // resident CTAs per SM of the single-view cull (<= 48 registers)

// Single-view streaming cull with direct streaming loads: each thread issues
// its kCullPT 16-byte loads for a pass up front (evict-first), then tests
// them two at a time on the paired FP32 pipes; resident warps hide each
// other's load latency.  No block-wide barrier: survivors go straight to
// global memory through per-warp slabs (slab_push; only each warp's last
// slab has unused slots, which are filled with kNoId and skipped by the setup
// stage), and the depth range is kept in registers and reduced once at the
// end.  PLAIN: van der Waals radii and no clip plane.
template <bool PLAIN, bool STAGE>
__global__ __launch_bounds__(kCullThreads, kCullCtasPerSm) void k_cull_direct(Geometry g, const float4 *__restrict__ X,
                                                                            ImageState *st,
                                                                            uint32_t *__restrict__ surv,
                                                                            float4 *__restrict__ stage) {
  pdl_enter();
  static_assert(kCullPT % 2 == 0, "atoms are tested in pairs");
  const ViewParams &vp = g.views[0];
  const long long n = g.n_atoms;
  constexpr int CH = kCullPT * kCullThreads;
  const int lane = threadIdx.x & 31;
  const unsigned lt = (1u << lane) - 1u;
  const long long cap = g.surv_cap;
  uint32_t slab = kNoId;
  int used = kSlab;
  float zlo = __int_as_float(0x7f800000), zhi = 0.0f;
  for (long long a0 = (long long)blockIdx.x * CH; a0 < n; a0 += (long long)gridDim.x * CH) {
    float4 a[kCullPT];
#pragma unroll
    for (int j = 0; j < kCullPT; ++j) {
      const long long i = a0 + j * kCullThreads + threadIdx.x;
      a[j] = i < n ? cull_load(X + i) : make_float4(0.0f, 0.0f, 0.0f, -1.0f);
    }
#pragma unroll
    for (int j = 0; j < kCullPT; j += 2) {
      const float4 p = a[j], q = a[j + 1];
      float2 vx, vy, vz, err;
      const float2 r = PLAIN ? make_float2(p.w, q.w) : make_float2(atom_radius(g, p.w), atom_radius(g, q.w));
      view_f32x2(vp, make_float2(p.x, q.x), make_float2(p.y, q.y), make_float2(p.z, q.z), vx, vy, vz, err);
      const float2 Rm = __fadd2_rn(r, err);
      bool k0, k1;
      cull_lean_x2(vp, vx, vy, vz, Rm, k0, k1);
      k0 = k0 && p.w >= 0.0f;
      k1 = k1 && q.w >= 0.0f;
      if (!PLAIN) {
        k0 = k0 && clip_keep(g, p.x, p.y, p.z);
        k1 = k1 && clip_keep(g, q.x, q.y, q.z);
      }
      if (k0) {
        zlo = fminf(zlo, vz.x - Rm.x);
        zhi = fmaxf(zhi, vz.x + Rm.x);
      }
      if (k1) {
        zlo = fminf(zlo, vz.y - Rm.y);
        zhi = fmaxf(zhi, vz.y + Rm.y);
      }
      if (STAGE) {  // survivors' records into device memory for setup and resolve (X is in host memory)
        if (k0) stage[a0 + j * kCullThreads + threadIdx.x] = p;
        if (k1) stage[a0 + (j + 1) * kCullThreads + threadIdx.x] = q;
      }
      slab_push(k0, (uint32_t)(a0 + j * kCullThreads + threadIdx.x), lane, lt, slab, used, &st[0].n_surv, surv, cap);
      slab_push(k1, (uint32_t)(a0 + (j + 1) * kCullThreads + threadIdx.x), lane, lt, slab, used, &st[0].n_surv, surv,
                cap);
    }
  }
  if (slab != kNoId)
    for (int i = used + lane; i < kSlab; i += 32)
      if ((long long)slab + i < cap) surv[slab + i] = kNoId;
  warp_minmax(zlo, zhi);
  if (lane == 0 && zhi > 0.0f) {
    atomicMin(&st[0].zlo_bits, __float_as_uint(fmaxf(zlo, 0.0f)));
    atomicMax(&st[0].zhi_bits, __float_as_uint(zhi));
  }
}

// CTAs of the single-view cull: one per pass of atoms, at most kCullCtasPerSm per SM.
static long long cull_one_ctas(long long n_atoms) {
  const long long chunk = (long long)kCullPT * kCullThreads;
  const long long chunks = (n_atoms + chunk - 1) / chunk;
  const long long most = (long long)kCullCtasPerSm * sm_count();
  return chunks < most ? (chunks > 0 ? chunks : 1) : most;
}

long long cull_survivor_slack(long long n_atoms) { return cull_one_ctas(n_atoms) * (kCullThreads / 32) * kSlab; }

// CTAs per frame of the multi-view direct cull: about kCullCtasPerSm per SM over all frames of a launch.
static int cull_multi_ctas(long long per_frame, int n_frames) {
  const long long chunk = (long long)kCullPT * kCullThreads;
  const long long chunks = (per_frame + chunk - 1) / chunk;
  long long want = ((long long)kCullCtasPerSm * sm_count() + n_frames - 1) / n_frames;
  if (want < 1) want = 1;
  const long long c = chunks < want ? chunks : want;
  return (int)(c > 0 ? c : 1);
}

long long cull_multi_slack(long long per_frame, int n_frames) {
  return (long long)cull_multi_ctas(per_frame, n_frames) * (kCullThreads / 32) * kSlab;
}

// Multi-view direct cull of a batch (frames x NV views, NV <= 4): each
// thread loads its kCullPT records of frame blockIdx.y once (the frame is read
// once for all its views), tests each pair against every view on the paired
// FP32 pipes, and appends the survivors of view v to image (frame, v) through
// per-warp slabs as the single-view cull does (no block barrier, no
// shared-memory staging; a warp's last slab per view is padded with kNoId).
template <bool PLAIN, int NV>
__global__ __launch_bounds__(kCullThreads, 4) void k_cull_multi(Geometry g, const float4 *__restrict__ frames,
                                                               const long long *__restrict__ counts, ImageState *st,
                                                               uint32_t *__restrict__ surv) {
  pdl_enter();
  const int frame = blockIdx.y;
  const long long n = counts ? counts[frame] : g.n_atoms;
  const float4 *X = frames + (long long)frame * g.stride;
  constexpr int CH = kCullPT * kCullThreads;
  const int lane = threadIdx.x & 31;
  const unsigned lt = (1u << lane) - 1u;
  const long long cap = g.surv_cap;
  uint32_t slab[NV];
  int used[NV];
  float zlo[NV], zhi[NV];
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    slab[v] = kNoId;
    used[v] = kSlab;
    zlo[v] = __int_as_float(0x7f800000);
    zhi[v] = 0.0f;
  }
  for (long long a0 = (long long)blockIdx.x * CH; a0 < n; a0 += (long long)gridDim.x * CH) {
    float4 a[kCullPT];
#pragma unroll
    for (int j = 0; j < kCullPT; ++j) {
      const long long i = a0 + j * kCullThreads + threadIdx.x;
      a[j] = i < n ? cull_load(X + i) : make_float4(0.0f, 0.0f, 0.0f, -1.0f);
    }
#pragma unroll
    for (int j = 0; j < kCullPT; j += 2) {
      const float4 p = a[j], q = a[j + 1];
      const float2 r = PLAIN ? make_float2(p.w, q.w) : make_float2(atom_radius(g, p.w), atom_radius(g, q.w));
      const bool in0 = p.w >= 0.0f && (PLAIN || clip_keep(g, p.x, p.y, p.z));
      const bool in1 = q.w >= 0.0f && (PLAIN || clip_keep(g, q.x, q.y, q.z));
      const uint32_t i0 = (uint32_t)(a0 + j * kCullThreads + threadIdx.x);
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        const ViewParams &vp = g.views[v];
        float2 vx, vy, vz, err;
        view_f32x2(vp, make_float2(p.x, q.x), make_float2(p.y, q.y), make_float2(p.z, q.z), vx, vy, vz, err);
        const float2 Rm = __fadd2_rn(r, err);
        bool k0, k1;
        cull_lean_x2(vp, vx, vy, vz, Rm, k0, k1);
        k0 = k0 && in0;
        k1 = k1 && in1;
        if (k0) {
          zlo[v] = fminf(zlo[v], vz.x - Rm.x);
          zhi[v] = fmaxf(zhi[v], vz.x + Rm.x);
        }
        if (k1) {
          zlo[v] = fminf(zlo[v], vz.y - Rm.y);
          zhi[v] = fmaxf(zhi[v], vz.y + Rm.y);
        }
        const int img = frame * g.n_views + v;
        uint32_t *sv = surv + (long long)img * cap;
        slab_push(k0, i0, lane, lt, slab[v], used[v], &st[img].n_surv, sv, cap);
        slab_push(k1, i0 + kCullThreads, lane, lt, slab[v], used[v], &st[img].n_surv, sv, cap);
      }
    }
  }
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    const int img = frame * g.n_views + v;
    uint32_t *sv = surv + (long long)img * cap;
    if (slab[v] != kNoId)
      for (int i = used[v] + lane; i < kSlab; i += 32)
        if ((long long)slab[v] + i < cap) sv[slab[v] + i] = kNoId;
    float lo = zlo[v], hi = zhi[v];
    warp_minmax(lo, hi);
    if (lane == 0 && hi > 0.0f) {
      atomicMin(&st[img].zlo_bits, __float_as_uint(fmaxf(lo, 0.0f)));
      atomicMax(&st[img].zhi_bits, __float_as_uint(hi));
    }
  }
}

// Bond cylinders (ball-and-stick, single frame, single view): the bounding
// sphere of each capped cylinder is culled like an atom.
__global__ __launch_bounds__(kCullThreads) void k_cull_bonds(Geometry g, const float4 *__restrict__ X,
                                                             const uint2 *__restrict__ pairs, ImageState *st,
                                                             uint32_t *__restrict__ surv) {
  pdl_enter();
  __shared__ uint32_t s_idx[kCullThreads];
  __shared__ int s_cnt;
  __shared__ unsigned int s_base;
  const ViewParams &vp = g.views[0];
  const int lane = threadIdx.x & 31;
  float zlo = __int_as_float(0x7f800000), zhi = 0.0f;
  for (long long base = (long long)blockIdx.x * kCullThreads; base < g.n_bonds;
       base += (long long)gridDim.x * kCullThreads) {
    if (threadIdx.x == 0) s_cnt = 0;
    __syncthreads();
    long long b = base + threadIdx.x;
    bool keep = false;
    if (b < g.n_bonds) {
      uint2 p = pairs[b];
      float4 A = X[p.x], B = X[p.y];
      float mx = 0.5f * (A.x + B.x), my = 0.5f * (A.y + B.y), mz = 0.5f * (A.z + B.z);
      float dx = B.x - A.x, dy = B.y - A.y, dz = B.z - A.z;
      float hl = 0.5f * sqrtf(dx * dx + dy * dy + dz * dz);
      float Rb = sqrtf(hl * hl + g.bond_radius * g.bond_radius) * 1.00001f;
      float vx, vy, vz, err;
      view_f32(vp, mx, my, mz, vx, vy, vz, err);
      err += 1.2e-7f * (fabsf(mx) + fabsf(my) + fabsf(mz)) + 1e-6f;
      keep = cull_lean(vp, vx, vy, vz, Rb + err) && clip_keep(g, A.x, A.y, A.z) && clip_keep(g, B.x, B.y, B.z);
      if (keep) {
        zlo = fminf(zlo, vz - Rb - err);
        zhi = fmaxf(zhi, vz + Rb + err);
      }
    }
    unsigned m = __ballot_sync(0xffffffffu, keep);
    if (m) {
      int leader = __ffs(m) - 1;
      int pos = 0;
      if (lane == leader) pos = atomicAdd(&s_cnt, __popc(m));
      pos = __shfl_sync(0xffffffffu, pos, leader);
      if (keep) s_idx[pos + __popc(m & ((1u << lane) - 1u))] = (uint32_t)(g.n_atoms + b);
    }
    __syncthreads();
    const int cnt = s_cnt;
    if (cnt > 0) {
      if (threadIdx.x == 0) s_base = atomicAdd(&st[0].n_surv, (unsigned)cnt);
      __syncthreads();
      for (int k = threadIdx.x; k < cnt; k += kCullThreads) surv[s_base + k] = s_idx[k];
    }
    __syncthreads();
  }
  warp_minmax(zlo, zhi);
  if (lane == 0 && zhi > 0.0f) {
    atomicMin(&st[0].zlo_bits, __float_as_uint(fmaxf(zlo, 0.0f)));
    atomicMax(&st[0].zhi_bits, __float_as_uint(zhi));
  }
}


// Depth-key range per image: [zlo, zhi] of the survivors, widened past the
// FP32 error of the cull and clamped to half the near plane.
// Depth-key range of image img from its survivors' range (the cull's
// atomics), widened by the FP32 rounding of those bounds.  Computed by every
// setup CTA of the image alike; CTA 0 stores it for the later stages.
__device__ __forceinline__ ImageState finalize_state(const Geometry &g, int img, ImageState s) {
  if (s.n_surv == 0u || s.zhi_bits == 0u) {
    s.valid = 0u;
    return s;
  }
  const ViewParams &v = g.views[img % g.n_views];
  float lo = __uint_as_float(s.zlo_bits), hi = __uint_as_float(s.zhi_bits);
  lo = fmaxf(lo - 4e-6f * fabsf(lo) - 1e-4f, 0.5f * v.znear);
  hi = hi + 4e-6f * fabsf(hi) + 1e-4f;
  if (!(hi > lo)) hi = lo + 1.0f;
  s.zlo = lo;
  s.S = kKeySpanF / (hi - lo);
  s.invS = (hi - lo) / kKeySpanF;
  s.valid = 1u;
  // occlusion pass: images with at least one survivor per kOcclPixels pixels (a depth complexity at which
  // most survivors are hidden)
  s.occl = (g.occl && !g.soft && (long long)s.n_surv * kOcclPixels >= g.pix_per_img) ? 1u : 0u;
  return s;
}

// ---------------------------------------------------------------- setup --

struct PrimGeom {
  Setup su;
  float rad;       // sphere radius or cylinder radius
  float3 A;        // cylinder axis (internal frame)
  float hl;        // cylinder half length (0 for spheres)
  float Rb;        // bounding radius
  float vx, vy, vz, err;  // FP32 view centre for the conservative box
};

// Precise setup of primitive `id` of image `img` (sphere or bond cylinder).
// `pre` (when non-null) is the already loaded record of atom `id`.
__device__ __forceinline__ PrimGeom prim_geom(const Geometry &g, const ViewParams &v, const float4 *X, const uint2 *bonds,
                                              uint32_t id, float zlo, float S, bool use_box_r,
                                              const float4 *pre = nullptr) {
  PrimGeom p;
  if ((long long)id < g.n_atoms || bonds == nullptr) {
    float4 a = pre ? *pre : X[id];
    float r = atom_radius(g, a.w);
    p.rad = r;
    p.hl = 0.0f;
    p.A = make_float3(0.0f, 0.0f, 0.0f);
    p.Rb = r;
    df dx, dy, dz;
    eye_offset(v, a, dx, dy, dz);
    p.su = precise_setup(v, dx, dy, dz, r, zlo, S);
    if (use_box_r) view_f32(v, a.x, a.y, a.z, p.vx, p.vy, p.vz, p.err);
  } else {
    uint2 pr = bonds[(long long)id - g.n_atoms];
    float4 A = X[pr.x], B = X[pr.y];
    df ax, ay, az, bx, by, bz;
    eye_offset(v, A, ax, ay, az);
    eye_offset(v, B, bx, by, bz);
    df mx = df_add(ax, bx), my = df_add(ay, by), mz = df_add(az, bz);
    mx.hi *= 0.5f; mx.lo *= 0.5f;
    my.hi *= 0.5f; my.lo *= 0.5f;
    mz.hi *= 0.5f; mz.lo *= 0.5f;
    float dx = B.x - A.x, dy = B.y - A.y, dz = B.z - A.z;
    float L = sqrtf(dx * dx + dy * dy + dz * dz);
    float inv = 1.0f / L;
    p.A = make_float3((v.R[0] * dx + v.R[1] * dy + v.R[2] * dz) * inv, (v.U[0] * dx + v.U[1] * dy + v.U[2] * dz) * inv,
                      (v.F[0] * dx + v.F[1] * dy + v.F[2] * dz) * inv);
    p.hl = 0.5f * L;
    p.rad = g.bond_radius;
    p.Rb = sqrtf(p.hl * p.hl + p.rad * p.rad) * 1.00001f;
    p.su = precise_setup(v, mx, my, mz, p.Rb, zlo, S);
    if (use_box_r) {
      float cx = 0.5f * (A.x + B.x), cy = 0.5f * (A.y + B.y), cz = 0.5f * (A.z + B.z);
      view_f32(v, cx, cy, cz, p.vx, p.vy, p.vz, p.err);
      p.err += 1.2e-7f * (fabsf(cx) + fabsf(cy) + fabsf(cz)) + 1e-6f;
    }
  }
  return p;
}

// Ray-cast primitive p at one pixel; s is relative to the reference depth.
__device__ __forceinline__ bool prim_hit(const PrimGeom &p, float3 o, const PixRay &r, float &s, int &kind,
                                         float &axial) {
  if (p.hl == 0.0f) {
    kind = 0;
    axial = 0.0f;
    return sphere_local(o, r, p.rad, s);
  }
  return cylinder_local(o, r, p.A, p.hl, p.rad, s, kind, axial);
}

// Ray-cast primitive p at every pixel of its candidate box, merging hits into the key plane K (one lane).
// One flat loop over the box's pixels: the lanes of a warp, whose boxes differ in shape, then run for the
// largest box's pixel count rather than for the most rows times the most columns.
__device__ __forceinline__ void splat_box(const Geometry &g, const ViewParams &v, const PrimGeom &p, const PixBox &box,
                                          float S, uint32_t id, unsigned long long *K) {
  const int npix = (box.x1 - box.x0 + 1) * (box.y1 - box.y0 + 1);
  int px = box.x0, py = box.y0;
  for (int i = 0; i < npix; ++i) {
    PixRay r = pix_ray(v, px, py);
    float3 o = local_o(p.su.u0.hi, p.su.u0.lo, p.su.v0.hi, p.su.v0.lo, p.su.k, p.su.dz, r);
    float sh;
    int kind;
    float axial;
    if (prim_hit(p, o, r, sh, kind, axial) && p.su.zr + sh >= v.znear)
      atomicMin(K + (long long)py * g.W + px, pack_key(p.su.keyc, sh, S, id));
    if (++px > box.x1) {
      px = box.x0;
      ++py;
    }
  }
}

// Setup occupancy: 4 CTAs per SM (63 registers, a few bytes spilled) and 8
// CTAs per SM of grid, measured best against 2 and 3 per SM and a 4-per-SM
// grid (4K overview 0.072 -> 0.065 ms, close view 0.97 -> 0.76 ms).
#ifndef VTX_SETUP_MINB
#define VTX_SETUP_MINB 4
#endif
#ifndef VTX_SETUP_GRID
#define VTX_SETUP_GRID 8
#endif
template <bool SOFT>
__global__ __launch_bounds__(256, VTX_SETUP_MINB) void k_setup(Geometry g, const float4 *__restrict__ frames,
                                               const uint2 *__restrict__ bonds, ImageState *st,
                                               const uint32_t *__restrict__ surv, unsigned long long *keys,
                                               PrimRec *recs, uint32_t *rec_img, uint2 *rec_box, uint32_t *rec_of,
                                               uint32_t *tile_count, Status *status, uint32_t cap_rec,
                                               const uint32_t *kept) {
  pdl_enter();
  const int img = blockIdx.y;
  const ImageState s = finalize_state(g, img, st[img]);
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    st[img].zlo = s.zlo;
    st[img].S = s.S;
    st[img].invS = s.invS;
    st[img].valid = s.valid;
  }
  if (!s.valid) return;
  // with the occlusion pass (kept != null) an occlusion image takes the survivors its test kept; every other
  // image takes all its survivors
  const bool kept_list = kept != nullptr && s.occl;
  const ViewParams &v = g.views[img % g.n_views];
  const int frame = img / g.n_views;
  const float4 *X = frames + (long long)frame * g.stride;
  const long long n = min((long long)(kept_list ? st[img].n_vis : s.n_surv), g.surv_cap);
  const uint32_t *sv = (kept_list ? kept : surv) + (long long)img * g.surv_cap;
  unsigned long long *K = keys + (long long)img * g.pix_per_img;
  const int lane = threadIdx.x & 31;
  const long long stride = (long long)gridDim.x * blockDim.x;
  // two-stage prefetch: the id two iterations ahead, the atom record one ahead
  const long long k0 = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const float4 zero4 = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
  uint32_t id_cur = k0 < n ? sv[k0] : 0u;
  uint32_t id_nxt = k0 + stride < n ? sv[k0 + stride] : 0u;
  float4 a_cur = (k0 < n && (long long)id_cur < g.n_atoms) ? X[id_cur] : zero4;
  for (long long k = k0; k - lane < n; k += stride) {  // the same trip count for the lanes of a warp
    const float4 a_nxt = (k + stride < n && (long long)id_nxt < g.n_atoms) ? X[id_nxt] : zero4;
    const uint32_t id_nn = k + 2 * stride < n ? sv[k + 2 * stride] : 0u;
    bool binned = false;
    PrimRec rec;
    PixBox box;
    uint2 rbox = make_uint2(0u, 0u);
    const uint32_t id = id_cur;
    const float4 a_here = a_cur;
    id_cur = id_nxt;
    a_cur = a_nxt;
    id_nxt = id_nn;
    if (k < n && id != kNoId) {
      const bool is_atom = (long long)id < g.n_atoms || bonds == nullptr;
      bool any = true;
      if (is_atom) {
        // candidate box from the FP32 view centre (no precise setup needed for it)
        const float r = atom_radius(g, a_here.w);
        float vx, vy, vz, err;
        view_f32(v, a_here.x, a_here.y, a_here.z, vx, vy, vz, err);
        any = lean_box(v, g.W, g.H, vx, vy, vz, cull_radius(g, v, r, vz) + err, box);
      }
      PrimGeom p;
      if (any) {
        p = prim_geom(g, v, X, bonds, id, s.zlo, s.S, !is_atom, &a_here);
        if (!is_atom) any = lean_box(v, g.W, g.H, p.vx, p.vy, p.vz, p.Rb + p.err, box);
      }
      if (any) {
        const long long npx = (long long)(box.x1 - box.x0 + 1) * (long long)(box.y1 - box.y0 + 1);
        if (!SOFT && npx <= g.splat_max) {
          splat_box(g, v, p, box, s.S, id, K);
        } else {
          binned = true;
          rec.u0h = p.su.u0.hi;
          rec.u0l = p.su.u0.lo;
          rec.v0h = p.su.v0.hi;
          rec.v0l = p.su.v0.lo;
          rec.zr = p.su.zr;
          rec.k = p.su.k;
          rec.dz = p.su.dz;
          rec.rad = p.rad;
          long long kc = p.su.keyc;
          if (SOFT) {
            // soft order key: the centre depth, clamped into the key range
            kc = kc - round_ll(p.su.dz * s.S);
            kc = kc < 0 ? 0 : (kc > kKeySpan ? kKeySpan : kc);
          }
          rec.key_lo = (uint32_t)((unsigned long long)kc & 0xffffffffull);
          rec.key_hi = (int)(kc >> 32);
          rec.id = id;
          rec.hl = p.hl;
          rec.ax = p.A.x;
          rec.ay = p.A.y;
          rec.az = p.A.z;
          rec.pad = 0.0f;
          int tx0 = box.x0 / g.tile_w, tx1 = box.x1 / g.tile_w, ty0 = box.y0 / g.tile_h, ty1 = box.y1 / g.tile_h;
          rbox = make_uint2((uint32_t)tx0 | ((uint32_t)ty0 << 16), (uint32_t)tx1 | ((uint32_t)ty1 << 16));
        }
      }
    }
    const unsigned m = __ballot_sync(0xffffffffu, binned);
    unsigned base = 0u;
    if (m && lane == __ffs(m) - 1) base = atomicAdd(&status->n_rec, (unsigned)__popc(m));
    base = __shfl_sync(0xffffffffu, base, m ? __ffs(m) - 1 : 0);
    bool counted = false;
    if (binned) {
      const unsigned slot = base + __popc(m & ((1u << lane) - 1u));
      if (slot < cap_rec) {
        recs[slot] = rec;
        rec_img[slot] = (uint32_t)img;
        rec_box[slot] = rbox;
        if (SOFT) rec_of[(long long)img * g.n_atoms + rec.id] = slot;
        counted = true;
      } else {
        atomicOr(&status->overflow, 2u);
      }
    }
    // per-tile counts: lanes adding to the same tile in the same step are merged (neighbouring survivors
    // share tiles), so a busy tile's counter takes one atomic per warp and step instead of one per record
    if (__any_sync(0xffffffffu, counted)) {
      const int tx0 = rbox.x & 0xffff, ty0 = rbox.x >> 16, tx1 = rbox.y & 0xffff, ty1 = rbox.y >> 16;
      const int nx = tx1 - tx0 + 1, nt = counted ? nx * (ty1 - ty0 + 1) : 0;
      const int maxnt = (int)__reduce_max_sync(0xffffffffu, (unsigned)nt);
      uint32_t *tc = tile_count + (long long)img * g.tiles_per_img;
      for (int q = 0; q < maxnt; ++q) {
        const int tile = q < nt ? (ty0 + q / nx) * g.tiles_x + tx0 + q % nx : -1;
        const unsigned peers = __match_any_sync(0xffffffffu, tile);
        if (tile >= 0 && lane == __ffs(peers) - 1) atomicAdd(tc + tile, (unsigned)__popc(peers));
      }
    }
  }
}

// ------------------------------------------------------- occlusion pass --
// Images with many survivors per pixel (a trajectory blob seen whole) spend most of their setup on spheres
// that lose every depth test.  The pass proves most of them hidden before their precise setup, from bound keys
// written into the (still clear) key plane itself:
//   k_occl_upper: every survivor in the front share of the image's depth range writes, at each pixel whose ray
//     certainly meets its sphere, a key above every key its hit there can have: the depth key of an FP32
//     upper bound of its entry depth, raised past the key rounding, with the id of no primitive (atomicMin).
//     The final key of that pixel, over all survivors, is then below the bound key, whichever survivors are
//     processed later, and it is a primitive's key: the bound keys never survive to the resolve.
//   k_occl_test: a survivor is dropped when every pixel of its candidate box holds a key whose depth part is
//     below the smallest depth key any of its hits could have; the others are listed for setup.
// Exact: a dropped sphere's key at every pixel of its box is above the final key there, so it is never the
// minimum of any pixel and the key planes are those of the plain pass, bit for bit.  (The sphere that holds a
// pixel's minimum is never dropped, as its key there would have to be above itself.)

// Survivors per lane per step of the occlusion kernels: a warp takes 128 consecutive list entries (coalesced
// loads of four independent items in flight) and reserves its output slots with one atomic per warp.
// Measured on the 1,024-image batch: 4 per lane 25.15 ms, 2 per lane 25.50, 8 per lane 25.75 ms.
#ifndef VTX_OCCL_ITEMS
#define VTX_OCCL_ITEMS 4
#endif
constexpr int kOcclItems = VTX_OCCL_ITEMS;

// Warp-wide placement of up to kOcclItems flagged items per lane: one atomicAdd on *counter for the warp's
// total; returns each item's slot in the list, in item-major order of the flags.
__device__ __forceinline__ void occl_slots(const bool (&f)[kOcclItems], unsigned *counter, int lane,
                                           unsigned (&slot)[kOcclItems]) {
  unsigned m[kOcclItems], tot = 0u;
#pragma unroll
  for (int j = 0; j < kOcclItems; ++j) {
    m[j] = __ballot_sync(0xffffffffu, f[j]);
    tot += (unsigned)__popc(m[j]);
  }
  unsigned base = 0u;
  if (lane == 0 && tot) base = atomicAdd(counter, tot);
  base = __shfl_sync(0xffffffffu, base, 0);
  const unsigned below = (1u << lane) - 1u;
#pragma unroll
  for (int j = 0; j < kOcclItems; ++j) {
    slot[j] = base + (unsigned)__popc(m[j] & below);
    base += (unsigned)__popc(m[j]);
  }
}

// Most pixels a sphere's box may have and still be tested, or write its bound keys (larger ones are kept and
// write none: the bounds stay valid, only weaker).
constexpr int kOcclMaxPixels = 64;
// Share of the image's depth range whose spheres (by their front) write bounds.  Spheres farther back seldom
// hold a pixel's smallest bound; leaving them out halves the writer's work.  Measured on the 1,024-image
// trajectory batch: every sphere 29.7 ms, front 70 % 27.5, 50 % 25.9, 35 % 25.1, 25 % 25.6 ms.
#ifndef VTX_OCCL_UPPER_FRONT
#define VTX_OCCL_UPPER_FRONT 0.35f
#endif
constexpr float kOcclUpperFront = VTX_OCCL_UPPER_FRONT;

// The bound key of a hit depth bound ub: the depth key of ub, raised past every rounding of the key of a hit at
// a depth below ub (the FP32 difference and product here, ~2e-7 of the key, and the hit's own key rounding,
// tens of keys: 4e-6 of the key plus 8192 keys), with the id of no primitive, so that a primitive's key with
// the same depth part is still below it.  Beyond the key range: the background key (no bound).
__device__ __forceinline__ unsigned long long bound_key(float ub, float zlo, float S) {
  float kf = fmaxf((ub - zlo) * S, 0.0f);
  kf = fmaf(kf, 4e-6f, kf) + 8192.0f;
  if (!(kf < 4294967040.0f)) return kBgKey;
  return ((unsigned long long)(uint32_t)ceilf(kf) << 32) | (unsigned long long)kNoId;
}

// Upper bounds of the entry depth of the sphere at FP32 view position (vx, vy, vz) (error err per component)
// with radius r, at the pixels whose rays certainly meet it, merged as bound keys into the key plane Ki.  At pixel ray
// u = (a, b, 1) and w = (vx - a vz, vy - b vz) (the centre's offset from the ray at the centre's depth), the
// centre's squared distance to the ray is d2 = |w|^2 - (w.u)^2 / |u|^2, the ray's closest point to the centre
// lies at depth tc = vz + (w.u) / |u|^2 and it enters the sphere at depth tc - sqrt((r^2 - d2) / |u|^2).
// With del = 2 err + 1e-6 vz covering the FP32 errors of w, d2 and tc, a pixel is written when d2 <= rr^2,
// rr = 0.999 r - 2 del: the ray's true distance is then below 0.999 r - del, so the hit test meets the sphere
// there whatever its own rounding, and the bound tc - sqrt((rr^2 - d2) / |u|^2) + 2 del + 1e-4 exceeds the true
// entry depth by at least 1e-4 A (rr^2 - d2 is below the true r^2 - d^2).
__device__ __forceinline__ void occl_upper_splat(const Geometry &g, const ViewParams &v, unsigned long long *Ki,
                                                 float vx, float vy, float vz, float err, float r, float zlo, float S) {
  if (!(vz > 2.0f * (r + err) + v.znear)) return;  // no sphere near the eye plane (its reference depth moves)
  const float del = 2.0f * err + 1e-6f * vz;
  const float rr = fmaf(r, 0.999f, -2.0f * del);
  if (!(rr > 0.0f)) return;
  PixBox box;
  {
    // the pixel centres within rr f / vz of the projected centre (there |w| <= rr in exact arithmetic): any
    // box is valid, since every written pixel passes the distance test below
    const float rz = 1.0f / vz, Rs = rr * v.f * rz;
    const float ux = fmaf(v.f, vx * rz, v.cxm), uy = fmaf(-v.f, vy * rz, v.cym);
    box.x0 = (int)fmaxf(ceilf(ux - Rs), 0.0f);
    box.x1 = (int)fminf(floorf(ux + Rs), (float)(g.W - 1));
    box.y0 = (int)fmaxf(ceilf(uy - Rs), 0.0f);
    box.y1 = (int)fminf(floorf(uy + Rs), (float)(g.H - 1));
    if (!(box.x0 <= box.x1 && box.y0 <= box.y1)) return;
  }
  const int npix = (box.x1 - box.x0 + 1) * (box.y1 - box.y0 + 1);
  if (npix > kOcclMaxPixels) return;
  const float rr2 = rr * rr, dU = fmaf(2.0f, del, 1e-4f);
  int px = box.x0, py = box.y0;
  for (int i = 0; i < npix; ++i) {
    const PixRay q = pix_ray(v, px, py);
    const float wx = fmaf(-q.a, vz, vx), wy = fmaf(-q.b, vz, vy);
    const float wu = fmaf(wx, q.a, wy * q.b);
    const float d2 = fmaf(-wu * wu, q.inv_uu, fmaf(wx, wx, wy * wy));
    if (d2 <= rr2) {
      const float tc = fmaf(wu, q.inv_uu, vz);
      const float sq = sqrt_approx((rr2 - d2) * q.inv_uu);
      atomicMin(Ki + (long long)py * g.W + px, bound_key(fmaf(-0.99999f, sq, tc) + dU, zlo, S));
    }
    if (++px > box.x1) {
      px = box.x0;
      ++py;
    }
  }
}

// A warp reads 128 consecutive survivors (four independent loads per lane in flight), keeps the writers in
// shared memory and then spreads their pixel loops over all 32 lanes: about a third of the survivors write,
// so a lane per survivor would leave most lanes idle during the loops.
__global__ __launch_bounds__(256) void k_occl_upper(Geometry g, const float4 *__restrict__ frames, ImageState *st,
                                                    const uint32_t *__restrict__ surv, unsigned long long *keys) {
  pdl_enter();
  __shared__ float4 s_c[8][32 * kOcclItems];  // per warp: the writers' (vx, vy, vz, err)
  __shared__ float s_r[8][32 * kOcclItems];   // and radii
  const int img = blockIdx.y;
  const ImageState s = finalize_state(g, img, st[img]);
  if (blockIdx.x == 0 && threadIdx.x == 0) st[img].occl = s.occl;
  if (!s.valid || !s.occl) return;
  const long long n = min((long long)s.n_surv, g.surv_cap);
  const ViewParams &v = g.views[img % g.n_views];
  const float4 *X = frames + (long long)(img / g.n_views) * g.stride;
  const uint32_t *sv = surv + (long long)img * g.surv_cap;
  unsigned long long *Ki = keys + (long long)img * g.pix_per_img;
  const float zf = s.zlo + kOcclUpperFront * (kKeySpanF * s.invS);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const long long warp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const long long warps = ((long long)gridDim.x * blockDim.x) >> 5;
  for (long long base = warp * 32 * kOcclItems; base < n; base += warps * 32 * kOcclItems) {
    uint32_t id[kOcclItems];
#pragma unroll
    for (int j = 0; j < kOcclItems; ++j) {
      const long long k = base + j * 32 + lane;
      id[j] = k < n ? sv[k] : kNoId;
    }
    float4 a[kOcclItems];
#pragma unroll
    for (int j = 0; j < kOcclItems; ++j)
      a[j] = (id[j] != kNoId && (long long)id[j] < g.n_atoms) ? X[id[j]] : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    bool wr[kOcclItems];
    float4 c[kOcclItems];
    float rad[kOcclItems];
#pragma unroll
    for (int j = 0; j < kOcclItems; ++j) {
      float vx, vy, vz, err;
      view_f32(v, a[j].x, a[j].y, a[j].z, vx, vy, vz, err);
      rad[j] = atom_radius(g, a[j].w);
      c[j] = make_float4(vx, vy, vz, err);
      wr[j] = id[j] != kNoId && (long long)id[j] < g.n_atoms && !(vz - rad[j] - err > zf);
    }
    unsigned total = 0u;
    const unsigned below = (1u << lane) - 1u;
#pragma unroll
    for (int j = 0; j < kOcclItems; ++j) {
      const unsigned m = __ballot_sync(0xffffffffu, wr[j]);
      if (wr[j]) {
        const unsigned slot = total + (unsigned)__popc(m & below);
        s_c[wid][slot] = c[j];
        s_r[wid][slot] = rad[j];
      }
      total += (unsigned)__popc(m);
    }
    __syncwarp();
    for (unsigned t = lane; t < total; t += 32) {
      const float4 q = s_c[wid][t];
      occl_upper_splat(g, v, Ki, q.x, q.y, q.z, q.w, s_r[wid][t], s.zlo, s.S);
    }
    __syncwarp();  // the slots are read before the next step refills them
  }
}

// Is the sphere at FP32 view position (vx, vy, vz) (error err) with radius r, candidate box `box`, hidden at
// every pixel of its box by the keys in Ki (bound keys or the background)?  lb: the smallest depth key any of its
// hits could have -- its front (vz - r, widened by the view error and by 2e-7 of the depths for the FP32
// rounding of these differences) mapped to keys, less 4e-6 relative plus 4096 keys for the rounding of the
// product, of the reference key and of the hit offset (tens of keys).  A pixel whose key's depth part is below
// lb can take no key of this sphere.  Only the depth words (the upper halves of the keys) are read; boxes of at
// most 4 x 4 pixels (the common case) load all of theirs at once.
__device__ __forceinline__ bool occl_hidden(const Geometry &g, const ViewParams &v, const ImageState &s,
                                            const unsigned long long *Ki, float vz, float err, float r,
                                            const PixBox &box) {
  if (!(vz > 2.0f * (r + err) + v.znear)) return false;
  float lb = (vz - err - r * 1.000002f - s.zlo - 2e-7f * (fabsf(vz) + fabsf(s.zlo))) * s.S;
  lb = lb - fabsf(lb) * 4e-6f - 4096.0f;
  if (!(lb > 0.0f)) return false;
  const uint32_t lbi = (uint32_t)fminf(floorf(lb), 4294967040.0f);  // lbi <= lb
  const int w = box.x1 - box.x0 + 1, h = box.y1 - box.y0 + 1;
  // the depth word of a key: its upper 32 bits (little-endian)
  const uint32_t *Db = reinterpret_cast<const uint32_t *>(Ki + (long long)box.y0 * g.W + box.x0) + 1;
  if (w <= 4 && h <= 4) {
    uint32_t kd[16];
#pragma unroll
    for (int dy = 0; dy < 4; ++dy)
#pragma unroll
      for (int dx = 0; dx < 4; ++dx) kd[dy * 4 + dx] = (dx < w && dy < h) ? Db[2 * ((long long)dy * g.W + dx)] : 0u;
    bool hidden = true;
#pragma unroll
    for (int q = 0; q < 16; ++q) hidden = hidden && kd[q] < lbi;
    return hidden;
  }
  if (w * h > kOcclMaxPixels) return false;
  for (int dy = 0; dy < h; ++dy)
    for (int dx = 0; dx < w; ++dx)
      if (!(Db[2 * ((long long)dy * g.W + dx)] < lbi)) return false;
  return true;
}

__global__ __launch_bounds__(256) void k_occl_test(Geometry g, const float4 *__restrict__ frames, ImageState *st,
                                                   const uint32_t *__restrict__ surv,
                                                   const unsigned long long *__restrict__ keys, uint32_t *kept) {
  pdl_enter();
  const int img = blockIdx.y;
  const ImageState s = finalize_state(g, img, st[img]);
  if (!s.valid || !s.occl) return;
  const long long n = min((long long)s.n_surv, g.surv_cap);
  const ViewParams &v = g.views[img % g.n_views];
  const float4 *X = frames + (long long)(img / g.n_views) * g.stride;
  const uint32_t *sv = surv + (long long)img * g.surv_cap;
  const unsigned long long *Ki = keys + (long long)img * g.pix_per_img;
  uint32_t *L = kept + (long long)img * g.surv_cap;
  const int lane = threadIdx.x & 31;
  const long long warp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const long long warps = ((long long)gridDim.x * blockDim.x) >> 5;
  for (long long base = warp * 32 * kOcclItems; base < n; base += warps * 32 * kOcclItems) {
    uint32_t id[kOcclItems];
    bool keep[kOcclItems];
#pragma unroll
    for (int j = 0; j < kOcclItems; ++j) {
      const long long k = base + j * 32 + lane;
      id[j] = k < n ? sv[k] : kNoId;
    }
#pragma unroll
    for (int j = 0; j < kOcclItems; ++j) {
      keep[j] = false;
      if (id[j] != kNoId && (long long)id[j] >= g.n_atoms) {
        keep[j] = true;  // not an atom record (the occlusion pass is for atoms): setup takes it as usual
      } else if (id[j] != kNoId) {
        const float4 a = X[id[j]];
        const float r = atom_radius(g, a.w);
        float vx, vy, vz, err;
        view_f32(v, a.x, a.y, a.z, vx, vy, vz, err);
        PixBox box;  // an empty box can change no pixel
        keep[j] = lean_box(v, g.W, g.H, vx, vy, vz, r + err, box) && !occl_hidden(g, v, s, Ki, vz, err, r, box);
      }
    }
    unsigned sk[kOcclItems];
    occl_slots(keep, &st[img].n_vis, lane, sk);
#pragma unroll
    for (int j = 0; j < kOcclItems; ++j)
      if (keep[j]) L[sk[j]] = id[j];
  }
}

// ----------------------------------------------------------------- scan --

__device__ __forceinline__ unsigned long long block_exclusive_scan_1024(unsigned long long v,
                                                                         unsigned long long *s_warp,
                                                                         unsigned long long &total) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  unsigned long long x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    unsigned long long y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) s_warp[wid] = x;
  __syncthreads();
  if (wid == 0) {
    unsigned long long w = lane < (int)(blockDim.x >> 5) ? s_warp[lane] : 0ull;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      unsigned long long y = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += y;
    }
    s_warp[lane] = w;
  }
  __syncthreads();
  unsigned long long off = wid > 0 ? s_warp[wid - 1] : 0ull;
  total = s_warp[(blockDim.x >> 5) - 1];
  __syncthreads();
  return off + x - v;
}

// Per-block exclusive scan of 4,096 tile counts; block totals to block_sums.
__global__ __launch_bounds__(1024) void k_scan_blocks(const uint32_t *__restrict__ cnt, long long n,
                                                      uint32_t *__restrict__ start, unsigned long long *block_sums) {
  pdl_enter();
  __shared__ unsigned long long s_warp[32];
  const long long base = (long long)blockIdx.x * kScanItems + (long long)threadIdx.x * 4;
  uint32_t c[4];
  unsigned long long sum = 0;
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    c[j] = base + j < n ? cnt[base + j] : 0u;
    sum += c[j];
  }
  unsigned long long total;
  unsigned long long ex = block_exclusive_scan_1024(sum, s_warp, total);
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    if (base + j < n) start[base + j] = (uint32_t)(ex > 0xffffffffull ? 0xffffffffull : ex);
    ex += c[j];
  }
  if (threadIdx.x == 0) block_sums[blockIdx.x] = total;
}

constexpr int kScanRounds = 32;                                 // values per lane in the one-CTA scan
static_assert(kScanSingleMax == 32LL * 32 * kScanRounds, "32 warps x 32 lanes x rounds");

// Exclusive scan of every tile count in one CTA (up to 1024 R tiles), listing
// the non-empty tiles for the raster stage on the way.  Warp w owns the
// contiguous segment [w S, (w+1) S), S = 32 R; each lane loads its R values
// up front (coalesced rows of 32), warps scan their rows with shuffles, and
// one pass over the 32 warp totals links the segments.  The launch picks the
// smallest R in {8, 16, 32} that covers the tiles: a 1080p frame's 8,160
// tiles take 8 rounds instead of the 32 a 4K frame needs.  The list is ordered
// longest first by classes of equal bit length of the count (a counting sort
// on the count's leading zeros), so that the kernels walking it start the
// longest tiles first and the short ones fill in behind them; the order
// within a class, like the order of the lists themselves, affects only
// scheduling.
template <int R>
__global__ __launch_bounds__(1024) void k_scan_single(const uint32_t *__restrict__ cnt, long long n,
                                                      uint32_t *__restrict__ start, uint32_t *__restrict__ cursor,
                                                      uint32_t *__restrict__ list, Status *status,
                                                      unsigned long long cap_entries, int skip_if_empty,
                                                      int list_empty) {
  pdl_enter();
  // hard edges: with no binned record every tile is empty; the raster reads
  // only the tile list (left empty by the set-up kernel) and the scatter has
  // nothing to place, so the scan has nothing to do
  if (skip_if_empty && status->n_rec == 0u) return;
  __shared__ unsigned long long s_wsum[32];
  // [0, 32): tiles per class (leading zeros of the count), then the class cursors; [32]: non-empty tiles;
  // [33]: cursor of the empty tiles, listed after all others when list_empty is set
  __shared__ unsigned int s_cls[34];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const long long seg = (long long)wid * 32 * R;
  if (threadIdx.x < 34) s_cls[threadIdx.x] = 0u;
  uint32_t v[R];
  unsigned long long wsum = 0;
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const long long i = seg + r * 32 + lane;
    v[r] = i < n ? cnt[i] : 0u;
  }
#pragma unroll
  for (int r = 0; r < R; ++r) wsum += v[r];
  __syncthreads();  // class counters cleared
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const int c = v[r] ? __clz(v[r]) : -1;
    const unsigned peers = __match_any_sync(0xffffffffu, c);
    if (c >= 0 && lane == __ffs(peers) - 1) atomicAdd(&s_cls[c], (unsigned)__popc(peers));
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) wsum += __shfl_xor_sync(0xffffffffu, wsum, o);
  if (lane == 0) s_wsum[wid] = wsum;
  __syncthreads();
  if (wid == 0) {
    unsigned long long x = s_wsum[lane];
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned long long y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    s_wsum[lane] = x - s_wsum[lane];  // exclusive
    if (lane == 31) {
      status->n_entries = x;
      start[n] = (uint32_t)(x > cap_entries ? cap_entries : x);
      if (x > cap_entries) atomicOr(&status->overflow, 4u);
    }
  } else if (wid == 1) {
    // class c starts after every class with fewer leading zeros (longer counts); s_cls[32] = tiles listed
    const unsigned c = s_cls[lane];
    unsigned y = c;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned t = __shfl_up_sync(0xffffffffu, y, o);
      if (lane >= o) y += t;
    }
    s_cls[lane] = y - c;
    if (lane == 31) {
      s_cls[32] = y;
      s_cls[33] = y;
    }
  }
  __syncthreads();
  unsigned long long carry = s_wsum[wid];
#pragma unroll
  for (int r = 0; r < R; ++r) {
    unsigned long long x = v[r];
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned long long y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    const unsigned long long ex = carry + x - v[r];
    const long long i = seg + r * 32 + lane;
    const bool ne = i < n && v[r] > 0u;
    if (i < n) {
      const uint32_t w = (uint32_t)(ex > cap_entries ? cap_entries : ex);
      start[i] = w;
      cursor[i] = w;
    }
    const int c = ne ? __clz(v[r]) : (list_empty && i < n ? 33 : -1);
    const unsigned peers = __match_any_sync(0xffffffffu, c);
    const int leader = __ffs(peers) - 1;
    unsigned base = 0u;
    if (c >= 0 && lane == leader) base = atomicAdd(&s_cls[c], (unsigned)__popc(peers));
    base = __shfl_sync(0xffffffffu, base, leader);
    if (c >= 0) list[base + __popc(peers & ((1u << lane) - 1u))] = (uint32_t)i;
    carry += __shfl_sync(0xffffffffu, x, 31);
  }
  if (threadIdx.x == 0) status->n_list = s_cls[32];
}

// Scan of the block totals (one CTA, loops when there are more than 1,024 blocks).
__global__ __launch_bounds__(1024) void k_scan_top(unsigned long long *block_sums, int nb, Status *status,
                                                   unsigned long long cap_entries) {
  pdl_enter();
  __shared__ unsigned long long s_warp[32];
  unsigned long long carry = 0;
  for (int b0 = 0; b0 < nb; b0 += 1024) {
    int i = b0 + threadIdx.x;
    unsigned long long v = i < nb ? block_sums[i] : 0ull;
    unsigned long long total;
    unsigned long long ex = block_exclusive_scan_1024(v, s_warp, total);
    if (i < nb) block_sums[i] = carry + ex;
    carry += total;
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    block_sums[nb] = carry;
    status->n_entries = carry;
    if (carry > cap_entries) atomicOr(&status->overflow, 4u);
  }
}

__global__ __launch_bounds__(1024) void k_scan_add(uint32_t *__restrict__ start, uint32_t *__restrict__ cursor,
                                                   long long n, const unsigned long long *__restrict__ block_sums,
                                                   unsigned long long cap_entries, const uint32_t *__restrict__ cnt,
                                                   uint32_t *__restrict__ list, Status *status) {
  pdl_enter();
  const long long base = (long long)blockIdx.x * kScanItems + (long long)threadIdx.x * 4;
  const unsigned long long off = block_sums[blockIdx.x];
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    long long i = base + j;
    bool ne = false;
    if (i < n) {
      unsigned long long v = off + start[i];
      uint32_t w = (uint32_t)(v > cap_entries ? cap_entries : v);
      start[i] = w;
      cursor[i] = w;
      ne = cnt[i] > 0u;
    }
    const unsigned m = __ballot_sync(0xffffffffu, ne);
    if (m) {
      const int leader = __ffs(m) - 1;
      unsigned b = 0u;
      if (lane == leader) b = atomicAdd(&status->n_list, (unsigned)__popc(m));
      b = __shfl_sync(0xffffffffu, b, leader);
      if (ne) list[b + __popc(m & ((1u << lane) - 1u))] = (uint32_t)i;
    }
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    unsigned long long tot = block_sums[gridDim.x];
    start[n] = (uint32_t)(tot > cap_entries ? cap_entries : tot);
  }
}

// -------------------------------------------------------------- scatter --

// Each lane takes one record; a warp walks its records' tiles in lockstep,
// four tile slots at a time.  Lanes that target the same tile in the same
// slot (neighbouring records share tiles) are merged with __match_any_sync:
// their leader reserves all their places with one atomicAdd, so the four
// slots' atomics are in flight together and the per-tile cursors see one
// atomic per warp instead of one per record.
template <bool SOFT>
__global__ __launch_bounds__(256) void k_scatter(Geometry g, const PrimRec *__restrict__ recs,
                                                 const uint32_t *__restrict__ rec_img,
                                                 const uint2 *__restrict__ rec_box,
                                                 const ImageState *__restrict__ st, const Status *__restrict__ status,
                                                 uint32_t cap_rec, uint32_t *tile_cursor,
                                                 unsigned long long *entries, unsigned long long cap_entries) {
  pdl_enter();
  const uint32_t n = min(status->n_rec, cap_rec);
  const int lane = threadIdx.x & 31;
  const unsigned lt = (1u << lane) - 1u;
  const uint32_t stride = gridDim.x * blockDim.x;
  for (uint32_t base = blockIdx.x * blockDim.x + (threadIdx.x & ~31u); base < n; base += stride) {
    const uint32_t r = base + (uint32_t)lane;
    unsigned long long key = 0ull;
    long long tile0 = 0;
    int nx = 1, nt = 0;
    if (r < n) {
      const PrimRec &q = recs[r];
      const int img = (int)rec_img[r];
      const uint2 bx = rec_box[r];
      if (SOFT) {
        key = ((unsigned long long)q.key_lo << 32) | (unsigned long long)q.id;
      } else {
        const float S = st[img].S;
        float Rb = q.hl == 0.0f ? q.rad : sqrtf(q.hl * q.hl + q.rad * q.rad);
        long long kmin = rec_key(q) - float_to_ll(ceilf((Rb + fabsf(q.dz)) * S * 1.000001f)) - 2;
        kmin = kmin < 0 ? 0 : (kmin > kKeySpan ? kKeySpan : kmin);
        key = ((unsigned long long)kmin << 32) | (unsigned long long)r;
      }
      const int tx0 = bx.x & 0xffff, ty0 = bx.x >> 16, tx1 = bx.y & 0xffff, ty1 = bx.y >> 16;
      nx = tx1 - tx0 + 1;
      nt = nx * (ty1 - ty0 + 1);
      tile0 = (long long)img * g.tiles_per_img + (long long)ty0 * g.tiles_x + tx0;
    }
    const int maxnt = __reduce_max_sync(0xffffffffu, (unsigned)nt);
    for (int k0 = 0; k0 < maxnt; k0 += 4) {
      unsigned peers[4];
      uint32_t got[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int k = k0 + u;
        const long long tile = k < nt ? tile0 + (long long)(k / nx) * g.tiles_x + (k % nx) : -1LL;
        peers[u] = __match_any_sync(0xffffffffu, (unsigned long long)tile);
        got[u] = 0u;
        if (k < nt && lane == __ffs(peers[u]) - 1) got[u] = atomicAdd(tile_cursor + tile, (unsigned)__popc(peers[u]));
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const uint32_t b0 = __shfl_sync(0xffffffffu, got[u], __ffs(peers[u]) - 1);
        if (k0 + u < nt) {
          const unsigned long long pos = (unsigned long long)b0 + (unsigned)__popc(peers[u] & lt);
          if (pos < cap_entries) entries[pos] = key;
        }
      }
    }
  }
}

// --------------------------------------------------------------- raster --

// Front-to-back order of one list segment by depth bucket (a one-pass
// counting sort in shared memory, replacing a full sort of the 64-bit
// entries).  The segment's nearest-depth keys [lo, hi] are cut into
// kRasterBuckets buckets by a monotone FP32 map, so every key of a bucket is
// <= every key of a later bucket.  Each entry is written to s_e as
// (smallest key of its bucket << 32 | record): that bound is non-decreasing
// along s_e and no later entry can be nearer than it, which is all the walk's
// early termination needs.  Order within a bucket follows shared-memory
// atomics; the visibility result (a minimum over all hits) does not depend
// on it.  src is the segment in global memory, read three times (L1 hits
// after the first).
constexpr int kRasterBuckets = 256;

template <int TW, int TH>
__device__ __forceinline__ uint32_t entry_box(const PrimRec *__restrict__ recs, uint32_t ri, int tx0, int ty0,
                                              float uu_max);

// While placing each entry, the final pass also stores its 16-bit pixel box (entry_box) beside it in s_box.
template <int TW, int TH>
__device__ __forceinline__ void bucket_order(const unsigned long long *__restrict__ src, int m,
                                             unsigned long long *s_e, uint16_t *s_off, uint32_t *s_cnt,
                                             uint32_t *s_lo, uint32_t *s_red, const PrimRec *__restrict__ recs,
                                             uint16_t *s_box, int tx0, int ty0, float uu_tile) {
  constexpr int NT = TW * TH;
  constexpr int NB = kRasterBuckets;
  static_assert(NB % NT == 0 && NT <= NB, "buckets per thread");
  constexpr int PER = NB / NT;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  uint32_t lo = 0xffffffffu, hi = 0u;
  for (int i = threadIdx.x; i < m; i += NT) {
    const uint32_t k = (uint32_t)(src[i] >> 32);
    lo = min(lo, k);
    hi = max(hi, k);
  }
  lo = __reduce_min_sync(0xffffffffu, lo);
  hi = __reduce_max_sync(0xffffffffu, hi);
#pragma unroll
  for (int j = 0; j < PER; ++j) {
    s_cnt[threadIdx.x * PER + j] = 0u;
    s_lo[threadIdx.x * PER + j] = 0xffffffffu;
  }
  if (threadIdx.x == 0) {
    s_red[0] = 0xffffffffu;
    s_red[1] = 0u;
  }
  __syncthreads();
  if (lane == 0) {
    atomicMin(s_red, lo);
    atomicMax(s_red + 1, hi);
  }
  __syncthreads();
  lo = s_red[0];
  hi = s_red[1];
  const float scale = (float)NB / ((float)(hi - lo) + 1.0f);
  for (int i = threadIdx.x; i < m; i += NT) {
    const uint32_t k = (uint32_t)(src[i] >> 32);
    const int b = min(NB - 1, (int)((float)(k - lo) * scale));
    s_off[i] = (uint16_t)atomicAdd(s_cnt + b, 1u);
    atomicMin(s_lo + b, k);
  }
  __syncthreads();
  // exclusive scan of the bucket counts: PER consecutive buckets per thread
  __shared__ uint32_t s_wt[NT / 32];
  uint32_t c[PER], sum = 0u;
#pragma unroll
  for (int j = 0; j < PER; ++j) {
    c[j] = s_cnt[threadIdx.x * PER + j];
    sum += c[j];
  }
  uint32_t inc = sum;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += y;
  }
  if (lane == 31) s_wt[wid] = inc;
  __syncthreads();
  uint32_t base = inc - sum;
  for (int w = 0; w < wid; ++w) base += s_wt[w];
#pragma unroll
  for (int j = 0; j < PER; ++j) {
    s_cnt[threadIdx.x * PER + j] = base;
    base += c[j];
  }
  __syncthreads();
  for (int i = threadIdx.x; i < m; i += NT) {
    const unsigned long long e = src[i];
    const uint32_t k = (uint32_t)(e >> 32);
    const int b = min(NB - 1, (int)((float)(k - lo) * scale));
    const uint32_t pos = s_cnt[b] + s_off[i];
    s_e[pos] = ((unsigned long long)s_lo[b] << 32) | (e & 0xffffffffull);
    s_box[pos] = (uint16_t)entry_box<TW, TH>(recs, (uint32_t)e, tx0, ty0, uu_tile);
  }
  __syncthreads();
}

constexpr int kListCap = 2048;

// A warp's 32-entry window is culled against the bounding rectangle
// [x0, x1] x [y0, y1] of its still-searching pixels (integer pixel indices).
// With the reference point at the bounding sphere's centre (dz = 0), the
// offset at the reference depth is o = k (du, -dv, 0), and the centre's
// distance to a pixel ray is >= |o| / |u| (Cauchy-Schwarz on the x, y part),
// so no ray of the rectangle meets the bounding sphere (radius Rb) when the
// pixel distance d from the projected centre exceeds Rb |u|_max / k.  The
// radius is widened (0.1 % plus 0.01 px plus 2e-7 of the coordinates) so that
// FP32 rounding never drops an entry the hit test would accept.
// Pixel radius about (cu, cv) outside which no ray with |u|^2 <= uu_max meets the bounding sphere.
__device__ __forceinline__ float raster_reach(float hl, float rad, float k, float cu, float cv, float uu_max) {
  const float rb2 = fmaf(hl, hl, rad * rad);
  const float rb = hl == 0.0f ? rad : rb2 * rsqrtf(rb2);
  return __fdividef(rb * uu_max * rsqrtf(uu_max), k) * 1.001f + 0.01f + 2e-7f * (fabsf(cu) + fabsf(cv));
}

__device__ __forceinline__ bool raster_keep(const PrimRec &p, unsigned x0, unsigned x1, unsigned y0, unsigned y1,
                                            float uu_max) {
  if (p.dz != 0.0f) return true;
  const float cu = p.u0h + p.u0l, cv = p.v0h + p.v0l;
  const float dx = fmaxf(fmaxf((float)x0 + 0.5f - cu, cu - ((float)x1 + 0.5f)), 0.0f);
  const float dy = fmaxf(fmaxf((float)y0 + 0.5f - cv, cv - ((float)y1 + 0.5f)), 0.0f);
  const float rt = raster_reach(p.hl, p.rad, p.k, cu, cv, uu_max);
  return !(dx * dx + dy * dy > rt * rt);
}

// The tile pixels an entry can reach, as a 16-bit box of tile-local indices (x0, x1, y0, y1 in XB, XB, YB, YB
// bits; x0 > x1 when it reaches none).  A pixel whose centre lies farther than the reach from the projected
// centre along x or along y is farther than the reach in the plane, so its ray cannot meet the bounding
// sphere; the box keeps every other pixel.  uu_max bounds |u|^2 over the whole tile.  Computed once per
// entry while the tile is ordered, it lets a warp skip, without loading their records, the entries that
// cannot reach any of its still-searching pixels.
template <int TW, int TH>
__device__ __forceinline__ uint32_t entry_box(const PrimRec *__restrict__ recs, uint32_t ri, int tx0, int ty0,
                                              float uu_max) {
  constexpr int XB = TW == 32 ? 5 : (TW == 16 ? 4 : 3), YB = TH == 16 ? 4 : 3;
  static_assert((1 << XB) == TW && (1 << YB) == TH && 2 * (XB + YB) <= 16, "tile shape");
  const PrimRec *pr = recs + ri;
  const float4 uv = __ldg(reinterpret_cast<const float4 *>(pr));      // u0h, u0l, v0h, v0l
  const float4 zk = __ldg(reinterpret_cast<const float4 *>(pr) + 1);  // zr, k, dz, rad
  const float hl = __ldg(&pr->hl);
  int x0 = 0, x1 = TW - 1, y0 = 0, y1 = TH - 1;
  if (zk.z == 0.0f) {
    const float cu = uv.x + uv.y, cv = uv.z + uv.w;
    const float rt = raster_reach(hl, zk.w, zk.y, cu, cv, uu_max);
    // pixel px is kept when |px + 0.5 - cu| <= rt; clamped to the tile in float first (no int overflow)
    const float lo_x = fmaxf(ceilf(cu - rt - 0.5f) - (float)tx0, 0.0f);
    const float hi_x = fminf(floorf(cu + rt - 0.5f) - (float)tx0, (float)(TW - 1));
    const float lo_y = fmaxf(ceilf(cv - rt - 0.5f) - (float)ty0, 0.0f);
    const float hi_y = fminf(floorf(cv + rt - 0.5f) - (float)ty0, (float)(TH - 1));
    if (!(lo_x <= hi_x && lo_y <= hi_y)) return (uint32_t)(TW - 1);  // x0 = TW - 1 > x1 = 0: no pixel
    x0 = (int)lo_x;
    x1 = (int)hi_x;
    y0 = (int)lo_y;
    y1 = (int)hi_y;
  }
  return (uint32_t)x0 | ((uint32_t)x1 << XB) | ((uint32_t)y0 << (2 * XB)) | ((uint32_t)y1 << (2 * XB + YB));
}

// Does the box meet the rectangle [x0, x1] x [y0, y1] (tile-local; empty when x0 > x1)?
template <int TW, int TH>
__device__ __forceinline__ bool box_meets(uint32_t b, int x0, int x1, int y0, int y1) {
  constexpr int XB = TW == 32 ? 5 : (TW == 16 ? 4 : 3), YB = TH == 16 ? 4 : 3;
  const int bx0 = (int)(b & (TW - 1)), bx1 = (int)((b >> XB) & (TW - 1));
  const int by0 = (int)((b >> (2 * XB)) & (TH - 1)), by1 = (int)((b >> (2 * XB + YB)) & (TH - 1));
  return bx0 <= bx1 && bx0 <= x1 && x0 <= bx1 && by0 <= y1 && y0 <= by1;
}

// Dynamic shared memory of the raster: the segment's ordered entries, then per warp two 32-record windows
// (the one being tested and the next one, filled by cp.async meanwhile), which also hold the bucket offsets
// while a segment is ordered, then the entries' 16-bit pixel boxes.
template <int NT>
__host__ __device__ constexpr size_t raster_windows() {
  return NT * 2 * sizeof(PrimRec) > kListCap * 2 ? NT * 2 * sizeof(PrimRec) : kListCap * 2;
}
template <int NT>
__host__ __device__ constexpr size_t raster_smem() {
  return kListCap * sizeof(unsigned long long) + raster_windows<NT>() + kListCap * sizeof(uint16_t);
}

// Copy the 64-byte records of the window entries [c0, c0 + 32) whose pixel boxes meet the rectangle
// [x0, x1] x [y0, y1] of the warp's still-searching pixels into this warp's window w (one record per lane,
// four 16-byte asynchronous copies) and close the lane's commit group (an empty group when the lane copies
// nothing, so every lane always has the same number of groups in flight).  Returns the warp's mask of copied
// entries: the others are neither loaded nor read, and a window with none is skipped without a wait.
template <int TW, int TH>
__device__ __forceinline__ unsigned raster_stage(const PrimRec *__restrict__ recs, const unsigned long long *s_e,
                                                 const uint16_t *s_box, int m, int c0, PrimRec *w, int lane, int x0,
                                                 int x1, int y0, int y1) {
  const bool take = c0 + lane < m && box_meets<TW, TH>(s_box[c0 + lane], x0, x1, y0, y1);
  if (take) {
    const char *src = reinterpret_cast<const char *>(recs + (uint32_t)s_e[c0 + lane]);
    char *dst = reinterpret_cast<char *>(w + lane);
#pragma unroll
    for (int b = 0; b < 64; b += 16) cp_async16(dst + b, src + b);
  }
  cp_async_commit();
  return __ballot_sync(0xffffffffu, take);
}

// |u|^2 bound over a whole tile: the ray slopes of its extreme columns and rows (pix_ray's operations, and
// every rounded step is monotone, so no pixel of the tile has a larger |u|^2).
template <int TW, int TH>
__device__ __forceinline__ float tile_uu_max(const ViewParams &v, int tx, int ty) {
  const float a0 = fabsf(__fmul_rn(__fsub_rn((float)(tx * TW) + 0.5f, v.cx), v.inv_f));
  const float a1 = fabsf(__fmul_rn(__fsub_rn((float)(tx * TW + TW - 1) + 0.5f, v.cx), v.inv_f));
  const float b0 = fabsf(__fmul_rn(__fsub_rn(v.cy, (float)(ty * TH) + 0.5f), v.inv_f));
  const float b1 = fabsf(__fmul_rn(__fsub_rn(v.cy, (float)(ty * TH + TH - 1) + 0.5f), v.inv_f));
  const float am = fmaxf(a0, a1), bm = fmaxf(b0, b1);
  return fmaf(am, am, fmaf(bm, bm, 1.0f));
}

#ifndef VTX_RASTER_PAIR
#define VTX_RASTER_PAIR 1  // test two window entries per step
#endif

// The packed key of record p's hit at pixel ray r, or the background key when the ray misses it.
__device__ __forceinline__ unsigned long long raster_hit(const PrimRec &p, const PixRay &r, float znear, float S) {
  const float3 o = local_o(p.u0h, p.u0l, p.v0h, p.v0l, p.k, p.dz, r);
  float s;
  bool hit;
  if (p.hl == 0.0f) {
    hit = sphere_local(o, r, p.rad, s);
  } else {
    int kind;
    float axial;
    hit = cylinder_local(o, r, make_float3(p.ax, p.ay, p.az), p.hl, p.rad, s, kind, axial);
  }
  return (hit && p.zr + s >= znear) ? pack_key(rec_key(p), s, S, p.id) : kBgKey;
}

// One CTA per tile at a time, the non-empty tiles longest first from a queue (as many CTAs as are resident):
// the tile's list is ordered by depth bucket with every entry's pixel box; then each warp walks it on its own.
template <int TW, int TH>
__global__ __launch_bounds__(TW *TH) void k_raster(Geometry g, const PrimRec *__restrict__ recs,
                                                   const unsigned long long *__restrict__ entries,
                                                   unsigned long long cap_entries,
                                                   const uint32_t *__restrict__ tile_count,
                                                   const uint32_t *__restrict__ tile_start,
                                                   const ImageState *__restrict__ st, unsigned long long *keys,
                                                   const uint32_t *__restrict__ tile_list, Status *status) {
  pdl_enter();
  constexpr int NT = TW * TH;
  static_assert(NT % 32 == 0, "whole warps per tile");
  extern __shared__ __align__(16) unsigned char raster_smem_raw[];
  unsigned long long *s_e = reinterpret_cast<unsigned long long *>(raster_smem_raw);
  unsigned char *s_raw = raster_smem_raw + kListCap * sizeof(unsigned long long);
  uint16_t *s_box = reinterpret_cast<uint16_t *>(s_raw + raster_windows<NT>());
  __shared__ uint32_t s_cnt[kRasterBuckets], s_lo[kRasterBuckets], s_red[2];
  __shared__ uint32_t s_li;
  PrimRec *s_w = reinterpret_cast<PrimRec *>(s_raw) + 2 * (threadIdx.x & ~31u);  // this warp's two windows
  const int lane = threadIdx.x & 31;
  const int lx = (int)(threadIdx.x % TW), ly = (int)(threadIdx.x / TW);  // tile-local pixel
  const uint32_t n_list = status->n_list;
  for (;;) {
    __syncthreads();  // every thread has read the previous tile's index
    if (threadIdx.x == 0) s_li = atomicAdd(&status->tile_next, 1u);
    __syncthreads();
    const uint32_t li = s_li;
    if (li >= n_list) break;
    const long long gt = tile_list[li];
    const int img = (int)(gt / g.tiles_per_img);
    const int t = (int)(gt % g.tiles_per_img);
    uint32_t cnt = tile_count[gt];
    if (cnt == 0u) continue;
    const uint32_t start = tile_start[gt];
    if ((unsigned long long)start >= cap_entries) continue;
    if ((unsigned long long)start + cnt > cap_entries) cnt = (uint32_t)(cap_entries - start);
    const ViewParams &v = g.views[img % g.n_views];
    const float S = st[img].S;
    const int tx = t % g.tiles_x, ty = t / g.tiles_x;
    const int px = tx * TW + lx, py = ty * TH + ly;
    const bool inside = px < g.W && py < g.H;
    const PixRay r = pix_ray(v, px, py);
    const float uu_max = __uint_as_float(__reduce_max_sync(0xffffffffu, __float_as_uint(r.uu)));
    const float uu_tile = tile_uu_max<TW, TH>(v, tx, ty);
    unsigned long long *K = keys + (long long)img * g.pix_per_img + (long long)py * g.W + px;
    unsigned long long best = inside ? *K : kBgKey;
    if (threadIdx.x == 0) atomicMax(&status->max_list, cnt);
    for (uint32_t seg = 0; seg < cnt; seg += kListCap) {
      const int m = (int)min((uint32_t)kListCap, cnt - seg);
      bucket_order<TW, TH>(entries + start + seg, m, s_e, reinterpret_cast<uint16_t *>(s_raw), s_cnt, s_lo, s_red,
                           recs, s_box, tx * TW, ty * TH, uu_tile);
      // each warp walks the sorted segment on its own, 32 entries at a time, the next window's records
      // arriving by cp.async while the current one is tested; only the entries whose pixel boxes meet the
      // rectangle of the warp's still-searching pixels are loaded; a pixel is finished once its hit is nearer
      // than the next entry's nearest possible depth
      bool done = !inside;
      int wb = 0;
      int rx0 = __reduce_min_sync(0xffffffffu, done ? TW : lx), rx1 = __reduce_max_sync(0xffffffffu, done ? -1 : lx);
      int ry0 = __reduce_min_sync(0xffffffffu, done ? TH : ly), ry1 = __reduce_max_sync(0xffffffffu, done ? -1 : ly);
      unsigned cur = raster_stage<TW, TH>(recs, s_e, s_box, m, 0, s_w, lane, rx0, rx1, ry0, ry1);
      for (int c0 = 0; c0 < m; c0 += 32, wb ^= 32) {
        if (!done && (uint32_t)(best >> 32) < (uint32_t)(s_e[c0] >> 32)) done = true;
        if (__all_sync(0xffffffffu, done)) break;
        rx0 = __reduce_min_sync(0xffffffffu, done ? TW : lx);
        rx1 = __reduce_max_sync(0xffffffffu, done ? -1 : lx);
        ry0 = __reduce_min_sync(0xffffffffu, done ? TH : ly);
        ry1 = __reduce_max_sync(0xffffffffu, done ? -1 : ly);
        const unsigned nxt = raster_stage<TW, TH>(recs, s_e, s_box, m, c0 + 32, s_w + (wb ^ 32), lane, rx0, rx1, ry0,
                                                  ry1);
        if (cur == 0u) {  // nothing of this window can reach the warp's pixels: no record was loaded
          cur = nxt;
          continue;
        }
        cp_async_wait<1>();  // this window's copies have landed (the next window's may still be in flight)
        __syncwarp();
        const PrimRec *win = s_w + wb;
        const unsigned x0 = (unsigned)(tx * TW + rx0), x1 = (unsigned)(tx * TW + rx1);
        const unsigned y0 = (unsigned)(ty * TH + ry0), y1 = (unsigned)(ty * TH + ry1);
        const bool keep = ((cur >> lane) & 1u) && raster_keep(win[lane], x0, x1, y0, y1, uu_max);
        const unsigned kept = __ballot_sync(0xffffffffu, keep);
        // two entries per step: their hit tests are independent chains the scheduler can interleave.  The
        // second is tested even when the first's bound would have finished the pixel after the first's
        // hit: one more candidate leaves the minimum unchanged, and the next step checks the bound again.
        for (unsigned b = kept; b != 0u;) {
          const int q1 = __ffs(b) - 1;
          b &= b - 1u;
          const int q2 = b != 0u ? __ffs(b) - 1 : -1;
          if (b != 0u) b &= b - 1u;
          if (done) continue;
          if ((uint32_t)(best >> 32) < (uint32_t)(s_e[c0 + q1] >> 32)) {
            done = true;
            continue;
          }
          const unsigned long long k1 = raster_hit(win[q1], r, v.znear, S);
          const unsigned long long k2 = (VTX_RASTER_PAIR && q2 >= 0) ? raster_hit(win[q2], r, v.znear, S) : kBgKey;
          if (!VTX_RASTER_PAIR && q2 >= 0) b |= 1u << q2;  // one entry per step: the second waits for the next
          best = k1 < best ? k1 : best;
          best = k2 < best ? k2 : best;
        }
        __syncwarp();  // every lane is done with this window before it is refilled
        cur = nxt;
      }
      cp_async_wait<0>();  // no copy may still target the windows when the next segment reuses them
      __syncthreads();
    }
    if (inside) *K = best;
  }
}

// -------------------------------------------------------------- resolve --

#ifndef VTX_SSAO_GROUP
#define VTX_SSAO_GROUP 4
#endif
#ifndef VTX_RESOLVE_MINB
#define VTX_RESOLVE_MINB 4
#endif
constexpr int kSsaoGroup = VTX_SSAO_GROUP;  // SSAO samples whose neighbour keys are fetched together
// Measured: 3 shading CTAs per SM beat 2 and 4 (2 starves the close view and
// the batch, 4 leaves too few CTAs for the background writes of the batch).
#ifndef VTX_SHADE_PER_SM
#define VTX_SHADE_PER_SM 3
#endif
#ifndef VTX_RESOLVE_2PASS
#define VTX_RESOLVE_2PASS 1
#endif

// A depth-key difference as float: the 32-bit conversion when it fits (the same rounding as the 64-bit one).
__device__ __forceinline__ float key_diff_f(long long d) {
  if (d >= -2147483647LL && d <= 2147483647LL) return __int2float_rn((int)d);
  return ll_to_float_wide(d);
}

__device__ __forceinline__ void resolve_pixel(const Geometry &g, const ShadeParams &sh, const float4 *__restrict__ frames,
                                              const uint8_t *__restrict__ elem, const uint2 *__restrict__ bonds,
                                              const ImageState *__restrict__ st,
                                              const unsigned long long *__restrict__ keys, const Outputs &out,
                                              int do_ssao, int img, int px, int py, unsigned long long key, Status *status) {
  const long long ppi = g.pix_per_img;
  {
    const long long p = (long long)py * g.W + px;
    const long long q = (long long)img * ppi + p;
    uint32_t id = (uint32_t)key;
    float *nrm = out.normal + (long long)img * 3 * ppi + p;
    float *rgb = out.rgb + (long long)img * 3 * ppi + p;
    // bounds check of the decoded id (a corrupted key): recorded in the status word, drawn as background
    if (id != kNoId && (long long)id >= g.n_atoms + g.n_bonds) {
      atomicOr(&status->overflow, 32u);
      id = kNoId;
    }
    if (id == kNoId) {
      out.depth[q] = __int_as_float(0x7f800000);
      out.id[q] = kNoId;
      nrm[0] = nrm[ppi] = nrm[2 * ppi] = 0.0f;
      rgb[0] = sh.bg[0];
      rgb[ppi] = sh.bg[1];
      rgb[2 * ppi] = sh.bg[2];
      if (out.ao) out.ao[q] = 1.0f;
      return;
    }
    const ViewParams &v = g.views[img % g.n_views];
    const ImageState s = st[img];
    const float4 *X = frames + (long long)(img / g.n_views) * g.stride;
    PrimGeom pg = prim_geom(g, v, X, bonds, id, s.zlo, s.S, false);
    const PixRay r = pix_ray(v, px, py);
    float3 o = local_o(pg.su.u0.hi, pg.su.u0.lo, pg.su.v0.hi, pg.su.v0.lo, pg.su.k, pg.su.dz, r);
    float sh_s = 0.0f, axial = 0.0f;
    int kind = 0;
    float3 ni;
    uint32_t atom = id;
    if (pg.hl == 0.0f) {
      float ou = fmaf(o.x, r.a, fmaf(o.y, r.b, o.z));
      float oo = fmaf(o.x, o.x, fmaf(o.y, o.y, o.z * o.z));
      float disc = fmaxf(fmaf(ou, ou, -r.uu * (oo - pg.rad * pg.rad)), 0.0f);
      sh_s = (-ou - sqrtf(disc)) / r.uu;
      float inv = 1.0f / pg.rad;
      ni = make_float3((o.x + sh_s * r.a) * inv, (o.y + sh_s * r.b) * inv, (o.z + sh_s) * inv);
    } else {
      cylinder_local(o, r, pg.A, pg.hl, pg.rad, sh_s, kind, axial);
      if (kind == 1) {
        float ua = fmaf(r.a, pg.A.x, fmaf(r.b, pg.A.y, pg.A.z));
        float oa = fmaf(o.x, pg.A.x, fmaf(o.y, pg.A.y, o.z * pg.A.z));
        float ax = oa + sh_s * ua;
        float inv = 1.0f / pg.rad;
        ni = make_float3((o.x + sh_s * r.a - ax * pg.A.x) * inv, (o.y + sh_s * r.b - ax * pg.A.y) * inv,
                         (o.z + sh_s - ax * pg.A.z) * inv);
      } else {
        float sg = kind == 2 ? 1.0f : -1.0f;
        ni = make_float3(sg * pg.A.x, sg * pg.A.y, sg * pg.A.z);
      }
      uint2 pr = bonds[(long long)id - g.n_atoms];
      atom = axial <= 0.0f ? pr.x : pr.y;
    }
    const float t = pg.su.zr + sh_s;
    const float3 n = make_float3(ni.x, ni.y, -ni.z);  // right-handed view frame
    const int e = elem ? (int)elem[atom] : 0;
    const float3 alb = make_float3(sh.palette[e][0], sh.palette[e][1], sh.palette[e][2]);
    float3 c = blinn_phong(sh, n, r, alb);
    float aof = 1.0f;
    if (do_ssao && sh.ssao_n > 0) {
      // tangent frame
      float3 a0 = fabsf(n.y) > 0.9f ? make_float3(1.0f, 0.0f, 0.0f) : make_float3(0.0f, 1.0f, 0.0f);
      float3 T = make_float3(n.y * a0.z - n.z * a0.y, n.z * a0.x - n.x * a0.z, n.x * a0.y - n.y * a0.x);
      float tinv = 1.0f / sqrtf(T.x * T.x + T.y * T.y + T.z * T.z);
      T.x *= tinv;
      T.y *= tinv;
      T.z *= tinv;
      float3 B = make_float3(n.y * T.z - n.z * T.y, n.z * T.x - n.x * T.z, n.x * T.y - n.y * T.x);
      const unsigned long long *Kimg = keys + (long long)img * ppi;
      const long long kP = (long long)(key >> 32);
      float occ = 0.0f;
      const float R = sh.ssao_radius;
      // samples in groups of kSsaoGroup: the group's neighbour-key loads are issued together
      for (int j0 = 0; j0 < sh.ssao_n; j0 += kSsaoGroup) {
        long long at[kSsaoGroup];
        float dls[kSsaoGroup];
#pragma unroll
        for (int u = 0; u < kSsaoGroup; ++u) {
          const int j = j0 + u;
          at[u] = -1;
          dls[u] = 0.0f;
          if (j < sh.ssao_n) {
            const float kx = sh.kernel[j][0], ky = sh.kernel[j][1], kz = sh.kernel[j][2];
            const float dx = R * (kx * T.x + ky * B.x + kz * n.x);
            const float dy = R * (kx * T.y + ky * B.y + kz * n.y);
            const float dzv = R * (kx * T.z + ky * B.z + kz * n.z);
            const float dl = -dzv;  // depth offset of the sample
            const float den = t + dl;
            dls[u] = dl;
            if (den > 0.0f) {
              const float fden = __fdiv_rn(v.f, den);  // one division for both offsets
              const float offx = fden * (dx - r.a * dl);
              const float offy = -fden * (dy - r.b * dl);
              const int ix = px + (int)floorf(0.5f + offx);
              const int iy = py + (int)floorf(0.5f + offy);
              if (ix >= 0 && iy >= 0 && ix < g.W && iy < g.H) at[u] = (long long)iy * g.W + ix;
            }
          }
        }
        unsigned long long kf[kSsaoGroup];
#pragma unroll
        for (int u = 0; u < kSsaoGroup; ++u) kf[u] = at[u] >= 0 ? Kimg[at[u]] : kBgKey;
#pragma unroll
        for (int u = 0; u < kSsaoGroup; ++u) {
          if ((uint32_t)kf[u] == kNoId) continue;
          const float dzf = key_diff_f((long long)(kf[u] >> 32) - kP) * s.invS;  // z_f - t
          if (dzf <= dls[u] - sh.ssao_bias) {
            const float adz = fabsf(dzf);
            occ += adz <= R ? 1.0f : R / adz;
          }
        }
      }
      aof = 1.0f - occ / (float)sh.ssao_n;
    }
    float3 col = make_float3(c.x * aof, c.y * aof, c.z * aof);
    if (sh.outline_depth > 0.0f) {
      // front side of a depth discontinuity: a 4-neighbour is background or deeper by more than outline_depth
      const unsigned long long *Kimg = keys + (long long)img * ppi;
      const long long kP = (long long)(key >> 32);
      const int nx[4] = {px - 1, px + 1, px, px};
      const int ny[4] = {py, py, py - 1, py + 1};
      bool edge = false;
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        if (nx[u] < 0 || ny[u] < 0 || nx[u] >= g.W || ny[u] >= g.H) continue;
        const unsigned long long kq = Kimg[(long long)ny[u] * g.W + nx[u]];
        if ((uint32_t)kq == kNoId || key_diff_f((long long)(kq >> 32) - kP) * s.invS > sh.outline_depth) edge = true;
      }
      if (edge) col = make_float3(sh.outline_color[0], sh.outline_color[1], sh.outline_color[2]);
    }
    if (sh.fog_density > 0.0f) {
      const float span = sh.fog_far - sh.fog_near;
      const float fz = span > 0.0f ? fminf(fmaxf((t - sh.fog_near) / span, 0.0f), 1.0f) : (t >= sh.fog_far ? 1.0f : 0.0f);
      const float fw = sh.fog_density * fz;
      col = make_float3(col.x + fw * (sh.bg[0] - col.x), col.y + fw * (sh.bg[1] - col.y), col.z + fw * (sh.bg[2] - col.z));
    }
    out.depth[q] = t;
    out.id[q] = id;
    nrm[0] = n.x;
    nrm[ppi] = n.y;
    nrm[2 * ppi] = n.z;
    rgb[0] = col.x;
    rgb[ppi] = col.y;
    rgb[2 * ppi] = col.z;
    if (out.ao) out.ao[q] = aof;
  }
}

// One 32x32 pixel block per CTA (4 rows per thread, the four keys loaded up front),
// blockIdx.z = image: no integer division per pixel.
__global__ __launch_bounds__(256, VTX_RESOLVE_MINB) void k_resolve(Geometry g, ShadeParams sh, const float4 *__restrict__ frames,
                                                 const uint8_t *__restrict__ elem, const uint2 *__restrict__ bonds,
                                                 const ImageState *__restrict__ st,
                                                 const unsigned long long *__restrict__ keys, Outputs out,
                                                 int do_ssao, Status *status) {
  pdl_enter();
  const int px = blockIdx.x * 32 + (threadIdx.x & 31);
  const int py0 = blockIdx.y * 32 + (threadIdx.x >> 5);
  const int img = blockIdx.z;
  if (px >= g.W) return;
  const unsigned long long *K = keys + (long long)img * g.pix_per_img;
  unsigned long long k0 = py0 < g.H ? K[(long long)py0 * g.W + px] : kBgKey;
  unsigned long long k1 = py0 + 8 < g.H ? K[(long long)(py0 + 8) * g.W + px] : kBgKey;
  unsigned long long k2 = py0 + 16 < g.H ? K[(long long)(py0 + 16) * g.W + px] : kBgKey;
  unsigned long long k3 = py0 + 24 < g.H ? K[(long long)(py0 + 24) * g.W + px] : kBgKey;
#pragma unroll 1
  for (int i = 0; i < 4; ++i) {  // one copy of the (large) pixel body: keys rotate through registers
    const unsigned long long key = k0;
    k0 = k1;
    k1 = k2;
    k2 = k3;
    const int py = py0 + 8 * i;
    if (py < g.H) resolve_pixel(g, sh, frames, elem, bonds, st, keys, out, do_ssao, img, px, py, key, status);
  }
}

// Two-pass resolve, pass 1: list the covered pixels (keys read, one atomic
// per warp).  Pass 2 (k_resolve_split) runs two kinds of CTA side by side:
// the first n_shade take the listed pixels one per thread through the long
// hit / shading / SSAO path (no background lanes idling beside a covered
// one), the others stream the constant outputs of background pixels (vector
// stores when VEC: four pixels per thread, every plane 16-byte aligned), so
// the latency-bound shading overlaps the memory-bound background writes.
// Measured against one pass (GB300, CUDA events): 1e8-atom 4K frame 0.102 ->
// 0.087 ms, close view 0.50 -> 0.34 ms, 1e5-atom 1080p 0.061 -> 0.031 ms;
// the 1,024-image trajectory batch (6 % coverage) is ~7 % slower in this
// stage.  A shared work queue interleaving both kinds and a plain two-pass
// form were measured too and were slower on the 4K frame.
template <bool VEC>
__global__ __launch_bounds__(256) void k_resolve_list(Geometry g, const unsigned long long *__restrict__ keys,
                                                      uint32_t *__restrict__ cov, uint32_t *__restrict__ mask,
                                                      Status *status) {
  pdl_enter();
  const long long total = g.pix_per_img * g.n_img;
  const int lane = threadIdx.x & 31;
  constexpr int P = VEC ? 4 : 1;
  const long long n_units = total / P;
  const long long stride = (long long)gridDim.x * blockDim.x;
  const long long n_iter = (n_units + stride - 1) / stride;
  for (long long it = 0; it < n_iter; ++it) {  // uniform trip count: every lane reaches the warp votes
    const long long u = it * stride + (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const bool live = u < n_units;
    const long long q0 = u * P;
    unsigned covered = 0u;
    if (live) {
      if (VEC) {
        const ulonglong2 a = *reinterpret_cast<const ulonglong2 *>(keys + q0);
        const ulonglong2 b = *reinterpret_cast<const ulonglong2 *>(keys + q0 + 2);
        covered = ((uint32_t)a.x != kNoId ? 1u : 0u) | ((uint32_t)a.y != kNoId ? 2u : 0u) |
                  ((uint32_t)b.x != kNoId ? 4u : 0u) | ((uint32_t)b.y != kNoId ? 8u : 0u);
      } else {
        covered = (uint32_t)keys[q0] != kNoId ? 1u : 0u;
      }
    }
    // coverage bits of the warp's 32 units (one word per pixel of a unit), for the background CTAs
#pragma unroll
    for (int v = 0; v < P; ++v) {
      const unsigned m = __ballot_sync(0xffffffffu, (covered >> v) & 1u);
      if (lane == 0 && live) mask[(u >> 5) * P + v] = m;
    }
    const int n_mine = __popc(covered);
    int incl = n_mine;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += y;
    }
    const int warp_total = __shfl_sync(0xffffffffu, incl, 31);
    if (warp_total == 0) continue;
    unsigned base = 0u;
    if (lane == 31) base = atomicAdd(&status->n_cov, (unsigned)warp_total);
    base = __shfl_sync(0xffffffffu, base, 31);
    unsigned at = base + (unsigned)(incl - n_mine);
#pragma unroll
    for (int v = 0; v < P; ++v)
      if (covered & (1u << v)) cov[at++] = (uint32_t)(q0 + v);
  }
}

template <bool VEC>
__global__ __launch_bounds__(256, VTX_RESOLVE_MINB) void k_resolve_split(
    Geometry g, ShadeParams sh, const float4 *__restrict__ frames, const uint8_t *__restrict__ elem,
    const uint2 *__restrict__ bonds, const ImageState *__restrict__ st, const unsigned long long *__restrict__ keys,
    Outputs out, int do_ssao, const uint32_t *__restrict__ cov, const uint32_t *__restrict__ mask,
    Status *status, int n_shade) {
  pdl_enter();
  const long long ppi = g.pix_per_img;
  if ((int)blockIdx.x < n_shade) {
    const unsigned n = status->n_cov;
    for (unsigned e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (unsigned)n_shade * blockDim.x) {
      const long long q = cov[e];
      const int img = (int)(q / ppi);
      const long long p = q - (long long)img * ppi;
      const int py = (int)(p / g.W), px = (int)(p - (long long)py * g.W);
      resolve_pixel(g, sh, frames, elem, bonds, st, keys, out, do_ssao, img, px, py, keys[q], status);
    }
    return;
  }
  constexpr int P = VEC ? 4 : 1;
  const long long n_units = ppi * g.n_img / P;
  const float inf = __int_as_float(0x7f800000);
  for (long long u = (long long)(blockIdx.x - n_shade) * blockDim.x + threadIdx.x; u < n_units;
       u += (long long)(gridDim.x - n_shade) * blockDim.x) {
    const long long q0 = u * P;
    unsigned covered = 0u;  // from the list pass's bits (1 bit per pixel) instead of the 8-byte keys
#pragma unroll
    for (int v = 0; v < P; ++v) covered |= ((mask[(u >> 5) * P + v] >> (u & 31)) & 1u) << v;
    const long long img = q0 / ppi, p = q0 - img * ppi;
    float *nrm = out.normal + img * 3 * ppi + p;
    float *rgb = out.rgb + img * 3 * ppi + p;
    if (VEC && covered == 0u) {
      const float4 z4 = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
      *reinterpret_cast<float4 *>(out.depth + q0) = make_float4(inf, inf, inf, inf);
      *reinterpret_cast<uint4 *>(out.id + q0) = make_uint4(kNoId, kNoId, kNoId, kNoId);
      *reinterpret_cast<float4 *>(nrm) = z4;
      *reinterpret_cast<float4 *>(nrm + ppi) = z4;
      *reinterpret_cast<float4 *>(nrm + 2 * ppi) = z4;
      *reinterpret_cast<float4 *>(rgb) = make_float4(sh.bg[0], sh.bg[0], sh.bg[0], sh.bg[0]);
      *reinterpret_cast<float4 *>(rgb + ppi) = make_float4(sh.bg[1], sh.bg[1], sh.bg[1], sh.bg[1]);
      *reinterpret_cast<float4 *>(rgb + 2 * ppi) = make_float4(sh.bg[2], sh.bg[2], sh.bg[2], sh.bg[2]);
      if (out.ao) *reinterpret_cast<float4 *>(out.ao + q0) = make_float4(1.0f, 1.0f, 1.0f, 1.0f);
    } else {
#pragma unroll
      for (int v = 0; v < P; ++v) {
        if (covered & (1u << v)) continue;
        out.depth[q0 + v] = inf;
        out.id[q0 + v] = kNoId;
        nrm[v] = nrm[ppi + v] = nrm[2 * ppi + v] = 0.0f;
        rgb[v] = sh.bg[0];
        rgb[ppi + v] = sh.bg[1];
        rgb[2 * ppi + v] = sh.bg[2];
        if (out.ao) out.ao[q0 + v] = 1.0f;
      }
    }
  }
}


// ------------------------------------------------------------ launchers --

static inline void ev_rec(StageEvents *e, int i, cudaStream_t st) {
  if (e && e->ev && i < e->n && ((e->mask >> i) & 1u)) cudaEventRecord(e->ev[i], st);
}

// Kernels of a frame are launched with programmatic stream serialisation:
// a kernel may be scheduled while its predecessor drains, and every kernel
// opens with pdl_enter(), which waits for the predecessor grid to complete
// (and its writes to be visible) before any memory access, then lets its
// successor start launching.  The stream order of all memory effects is
// unchanged; the launch latency and prologue of each kernel overlap the
// previous kernel's tail.
template <typename... P, typename... A>
static cudaError_t launch_pdl(void (*k)(P...), dim3 grid, int block, size_t smem, cudaStream_t st, A... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = dim3((unsigned)block);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k, static_cast<P>(args)...);
}

#ifndef VTX_CLEAR_MEMSET
#define VTX_CLEAR_MEMSET 1  // clear a batch's key planes with a memset instead of the clear kernel's stores
#endif

// Shared binning front end: init, cull, finalize, setup (+splat), scan, scatter.
cudaError_t run_binning(const Geometry &g, const Scene &sc, const Scratch &s, cudaStream_t st, StageEvents *evs,
                        bool soft) {
  const int sms = sm_count();
  const long long n_tiles = (long long)g.n_img * g.tiles_per_img;
  const bool occl = g.occl && !soft && s.defer;
  {
    // the background key has every bit set, so the key planes of a batch are cleared by a byte memset
    // (batch 30.9 -> 29.3 ms) instead of the clear kernel's stores; a single frame keeps the kernel, whose
    // launch overlaps its neighbours' (the memset slowed the 1e5-atom 1080p frame 0.081 -> 0.083 ms)
    const long long all_keys = soft ? 0 : g.pix_per_img * g.n_img;
    const bool fill = VTX_CLEAR_MEMSET && g.n_img > 1 && all_keys > 0;
    const long long n_keys = fill ? 0 : all_keys;
    if (fill) {
      static_assert(kBgKey == ~0ull, "a byte fill of 0xff gives the background key");
      cudaMemsetAsync(s.keys, 0xff, sizeof(unsigned long long) * (size_t)all_keys, st);
    }
    long long want = n_keys / 2 > n_tiles ? n_keys / 2 : n_tiles;
    want = want > g.n_img ? want : g.n_img;
    const long long blocks = (want + 255) / 256;
    const int gc = (int)(blocks < 16LL * sms ? (blocks > 0 ? blocks : 1) : 16LL * sms);
    launch_pdl(k_clear, gc, 256, 0, st, s.state, g.n_img, s.status, s.tile_count, n_tiles, s.keys, n_keys);
  }
  ev_rec(evs, 0, st);
  {
    static bool attr = false;
    if (!attr) {
      cudaFuncSetAttribute(k_cull_atoms<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kCullSmem);
      cudaFuncSetAttribute(k_cull_atoms<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kCullSmem);
      attr = true;
    }
    // five resident CTAs per SM in total, spread over the frames of a batch
    const long long per_frame = sc.counts ? g.stride : g.n_atoms;
    const long long chunks = (per_frame + kChunk - 1) / kChunk;
    long long want = (5LL * sms + g.n_frames - 1) / g.n_frames;
    if (want < 1) want = 1;
    int bx = (int)(chunks < want ? (chunks > 0 ? chunks : 1) : want);
    // few chunks (a small system seen from many views): one view per CTA
    const int vg = (g.n_views > 1 && (long long)bx * g.n_frames < 2LL * sms) ? g.n_views : 1;
    dim3 grid(bx, g.n_frames, vg);
    if (g.n_views == 1 && g.n_frames == 1 && sc.counts == nullptr && !g.soft) {
      const int b1 = (int)cull_one_ctas(g.n_atoms);
      const bool plain = g.mode == 0 && !g.clip_on;
      if (sc.stage && plain)
        launch_pdl(k_cull_direct<true, true>, b1, kCullThreads, 0, st, g, sc.frames, s.state, s.surv, sc.stage);
      else if (sc.stage)
        launch_pdl(k_cull_direct<false, true>, b1, kCullThreads, 0, st, g, sc.frames, s.state, s.surv, sc.stage);
      else if (plain)
        launch_pdl(k_cull_direct<true, false>, b1, kCullThreads, 0, st, g, sc.frames, s.state, s.surv, nullptr);
      else
        launch_pdl(k_cull_direct<false, false>, b1, kCullThreads, 0, st, g, sc.frames, s.state, s.surv, nullptr);
    } else if (!g.soft && g.n_views <= 4 && g.surv_cap >= per_frame + cull_multi_slack(per_frame, g.n_frames)) {
      // a batch (frames x up to 4 views): the barrier-free multi-view cull
      const dim3 gm(cull_multi_ctas(per_frame, g.n_frames), g.n_frames);
      const bool plain = g.mode == 0 && !g.clip_on;
      switch (g.n_views * 2 + (plain ? 1 : 0)) {
        case 2: launch_pdl(k_cull_multi<false, 1>, gm, kCullThreads, 0, st, g, sc.frames, sc.counts, s.state, s.surv); break;
        case 3: launch_pdl(k_cull_multi<true, 1>, gm, kCullThreads, 0, st, g, sc.frames, sc.counts, s.state, s.surv); break;
        case 4: launch_pdl(k_cull_multi<false, 2>, gm, kCullThreads, 0, st, g, sc.frames, sc.counts, s.state, s.surv); break;
        case 5: launch_pdl(k_cull_multi<true, 2>, gm, kCullThreads, 0, st, g, sc.frames, sc.counts, s.state, s.surv); break;
        case 6: launch_pdl(k_cull_multi<false, 3>, gm, kCullThreads, 0, st, g, sc.frames, sc.counts, s.state, s.surv); break;
        case 7: launch_pdl(k_cull_multi<true, 3>, gm, kCullThreads, 0, st, g, sc.frames, sc.counts, s.state, s.surv); break;
        case 8: launch_pdl(k_cull_multi<false, 4>, gm, kCullThreads, 0, st, g, sc.frames, sc.counts, s.state, s.surv); break;
        default: launch_pdl(k_cull_multi<true, 4>, gm, kCullThreads, 0, st, g, sc.frames, sc.counts, s.state, s.surv); break;
      }
    } else if (g.n_views == 1) {
      launch_pdl(k_cull_atoms<true>, grid, kCullThreads, kCullSmem, st, g, sc.frames, sc.counts, s.state, s.surv, s.status);
    } else {
      launch_pdl(k_cull_atoms<false>, grid, kCullThreads, kCullSmem, st, g, sc.frames, sc.counts, s.state, s.surv, s.status);
    }
    if (g.n_bonds > 0 && sc.bonds) {  // n_bonds is zero unless the representation draws bonds
      long long bb = (g.n_bonds + kCullThreads - 1) / kCullThreads;
      int gb = (int)(bb < 8LL * sms ? bb : 8LL * sms);
      launch_pdl(k_cull_bonds, gb, kCullThreads, 0, st, g, sc.frames, sc.bonds, s.state, s.surv);
    }
  }
  ev_rec(evs, 1, st);
  {
    int bx = g.n_img >= 64 ? VTX_SETUP_BATCH_CTAS : (VTX_SETUP_GRID * sms + g.n_img - 1) / g.n_img;
    dim3 grid(bx, g.n_img);
    if (soft)
      launch_pdl(k_setup<true>, grid, 256, 0, st, g, sc.frames, sc.bonds, s.state, s.surv, s.keys, s.recs, s.rec_img,
                                          s.rec_box, s.rec_of, s.tile_count, s.status, s.cap_rec, nullptr);
    else if (!occl)
      launch_pdl(k_setup<false>, grid, 256, 0, st, g, sc.stage ? sc.stage : sc.frames, sc.bonds, s.state, s.surv, s.keys,
                                           s.recs, s.rec_img, s.rec_box, s.rec_of, s.tile_count, s.status,
                                           s.cap_rec, nullptr);
    else {
      // occlusion pass (images that do not take it run all their survivors in setup): depth bounds, test,
      // setup of the kept survivors
      const float4 *Xs = sc.stage ? sc.stage : sc.frames;
      launch_pdl(k_occl_upper, grid, 256, 0, st, g, Xs, s.state, s.surv, s.keys);
      launch_pdl(k_occl_test, grid, 256, 0, st, g, Xs, s.state, s.surv, s.keys, s.defer);
      launch_pdl(k_setup<false>, grid, 256, 0, st, g, Xs, sc.bonds, s.state, s.surv, s.keys, s.recs, s.rec_img,
                 s.rec_box, s.rec_of, s.tile_count, s.status, s.cap_rec, s.defer);
    }
  }
  ev_rec(evs, 2, st);
  {
    if (n_tiles <= kScanSingleMax) {
      const int skip = soft ? 0 : 1;
      if (n_tiles <= 1024LL * 8)
        launch_pdl(k_scan_single<8>, 1, 1024, 0, st, s.tile_count, n_tiles, s.tile_start, s.tile_cursor, s.tile_list,
                                             s.status, s.cap_entries, skip, 1 - skip);
      else if (n_tiles <= 1024LL * 16)
        launch_pdl(k_scan_single<16>, 1, 1024, 0, st, s.tile_count, n_tiles, s.tile_start, s.tile_cursor, s.tile_list,
                                              s.status, s.cap_entries, skip, 1 - skip);
      else
        launch_pdl(k_scan_single<kScanRounds>, 1, 1024, 0, st, s.tile_count, n_tiles, s.tile_start, s.tile_cursor,
                                                       s.tile_list, s.status, s.cap_entries, skip, 1 - skip);
    } else {
      int nb = (int)((n_tiles + kScanItems - 1) / kScanItems);
      unsigned long long *bs = reinterpret_cast<unsigned long long *>(s.block_sums);
      launch_pdl(k_scan_blocks, nb, 1024, 0, st, s.tile_count, n_tiles, s.tile_start, bs);
      launch_pdl(k_scan_top, 1, 1024, 0, st, bs, nb, s.status, s.cap_entries);
      launch_pdl(k_scan_add, nb, 1024, 0, st, s.tile_start, s.tile_cursor, n_tiles, bs, s.cap_entries, s.tile_count,
                                      s.tile_list, s.status);
    }
  }
  ev_rec(evs, 3, st);
  if (soft)
    launch_pdl(k_scatter<true>, 4 * sms, 256, 0, st, g, s.recs, s.rec_img, s.rec_box, s.state, s.status, s.cap_rec,
                                             s.tile_cursor, s.entries, s.cap_entries);
  else
    launch_pdl(k_scatter<false>, 4 * sms, 256, 0, st, g, s.recs, s.rec_img, s.rec_box, s.state, s.status, s.cap_rec,
                                              s.tile_cursor, s.entries, s.cap_entries);
  ev_rec(evs, 4, st);
  return cudaGetLastError();
}

cudaError_t run_frame_pipeline(const Geometry &g, const ShadeParams &sh, const Scene &sc, const Scratch &s,
                               const Outputs &out, bool ssao, cudaStream_t st, StageEvents *evs) {
  cudaError_t e = run_binning(g, sc, s, st, evs, false);
  if (e != cudaSuccess) return e;
  const float4 *Xr = sc.stage ? sc.stage : sc.frames;  // winners are survivors: staged when staging is on
  const long long n_tiles = (long long)g.n_img * g.tiles_per_img;
  // raster CTAs: as many as are resident at once (the tile queue balances them), never more than tiles
  static int per_sm[3] = {0, 0, 0};
  static bool rattr = false;
  if (!rattr) {
    cudaFuncSetAttribute(k_raster<16, 16>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)raster_smem<256>());
    cudaFuncSetAttribute(k_raster<32, 8>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)raster_smem<256>());
    cudaFuncSetAttribute(k_raster<8, 8>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)raster_smem<64>());
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm[0], k_raster<16, 16>, 256, raster_smem<256>());
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm[1], k_raster<32, 8>, 256, raster_smem<256>());
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm[2], k_raster<8, 8>, 64, raster_smem<64>());
    for (int &q : per_sm) q = q > 0 ? q : 1;
    rattr = true;
  }
  const int shape = (g.tile_w == 16 && g.tile_h == 16) ? 0 : ((g.tile_w == 32 && g.tile_h == 8) ? 1 : 2);
  const long long resident = (long long)per_sm[shape] * sm_count();
  const unsigned rgrid = (unsigned)(n_tiles < resident ? (n_tiles > 0 ? n_tiles : 1) : resident);
  if (shape == 0)
    launch_pdl(k_raster<16, 16>, rgrid, 256, raster_smem<256>(), st, g, s.recs, s.entries, s.cap_entries,
               s.tile_count, s.tile_start, s.state, s.keys, s.tile_list, s.status);
  else if (shape == 1)
    launch_pdl(k_raster<32, 8>, rgrid, 256, raster_smem<256>(), st, g, s.recs, s.entries, s.cap_entries,
               s.tile_count, s.tile_start, s.state, s.keys, s.tile_list, s.status);
  else
    launch_pdl(k_raster<8, 8>, rgrid, 64, raster_smem<64>(), st, g, s.recs, s.entries, s.cap_entries,
               s.tile_count, s.tile_start, s.state, s.keys, s.tile_list, s.status);
  ev_rec(evs, 5, st);
  if (sc.dbg_corrupt_key && s.keys) cudaMemsetAsync(s.keys, 0x7f, sizeof(unsigned long long), st);  // test hook
  if (VTX_RESOLVE_2PASS && s.cov_list) {
    const int sms = sm_count();
    const long long total = g.pix_per_img * g.n_img;
    const bool vec = (g.pix_per_img % 4) == 0 && ((uintptr_t)out.depth | (uintptr_t)out.id | (uintptr_t)out.normal |
                                                  (uintptr_t)out.rgb | (uintptr_t)(out.ao ? out.ao : out.depth)) % 16 == 0;
    const long long units = vec ? total / 4 : total;
    const long long want = (units + 255) / 256;
    const int gl = (int)(want < 16LL * sms ? (want > 0 ? want : 1) : 16LL * sms);
    // shading CTAs first (they start at once and stay resident), background CTAs behind them
    const int n_shade = VTX_SHADE_PER_SM * sms;
    const int gb = (int)(want < 8LL * sms ? (want > 0 ? want : 1) : 8LL * sms);
    if (vec) {
      launch_pdl(k_resolve_list<true>, gl, 256, 0, st, g, s.keys, s.cov_list, s.cov_mask, s.status);
      ev_rec(evs, 6, st);
      launch_pdl(k_resolve_split<true>, n_shade + gb, 256, 0, st, g, sh, Xr, sc.elem, sc.bonds, s.state, s.keys, out,
                                                            ssao ? 1 : 0, s.cov_list, s.cov_mask, s.status, n_shade);
    } else {
      launch_pdl(k_resolve_list<false>, gl, 256, 0, st, g, s.keys, s.cov_list, s.cov_mask, s.status);
      ev_rec(evs, 6, st);
      launch_pdl(k_resolve_split<false>, n_shade + gb, 256, 0, st, g, sh, Xr, sc.elem, sc.bonds, s.state, s.keys, out,
                                                             ssao ? 1 : 0, s.cov_list, s.cov_mask, s.status, n_shade);
    }
  } else {
    dim3 grid((g.W + 31) / 32, (g.H + 31) / 32, g.n_img);
    launch_pdl(k_resolve, grid, 256, 0, st, g, sh, Xr, sc.elem, sc.bonds, s.state, s.keys, out, ssao ? 1 : 0,
               s.status);
    ev_rec(evs, 6, st);
  }
  ev_rec(evs, 7, st);
  return cudaGetLastError();
}

}  // namespace vtx
