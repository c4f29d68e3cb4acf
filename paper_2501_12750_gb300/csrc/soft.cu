// soft.cu -- soft-edge (differentiable) sphere renderer, forward and backward.
//
// Per pixel, the spheres whose signed pixel distance to their silhouette is
// at least -4 px are composited front to back in centre-depth order (ties:
// smaller id):
//   delta = (r - sqrt(rho^2 + 1e-12)) f / z_c        (rho: centre-to-ray distance)
//   alpha = min(0.99, sigmoid(delta / sigma))
//   g     = sqrt(max(r^2 - rho^2, 0) + eta^2) - eta,  eta = 0.05 r
//   t_i   = t_c - g / |u|         (smoothed entry depth; t_c = closest approach)
//   n_i   = (t_i u - C) / r
//   w_i = alpha_i T_i, T_{i+1} = T_i (1 - alpha_i), stop once T < 1e-4;
//   coverage = sum w_i, depth = sum w_i t_i, normal = sum w_i n_i.
// Binning (cull with 4 px dilation, precise setup, per-tile counting sort)
// is shared with the hard-edge path; each tile CTA (tiles longest first)
// sorts its list by (centre depth key, id) in shared memory (bucket pass plus
// per-bucket insertion sort; in global memory for lists longer than shared
// memory holds) and writes it back, then each warp walks the sorted list on
// its own, staging 32 entries at a time with their per-sphere constants
// (f / z_c, 1 / r and a bound on rho^2 that rejects most entries before any
// square root or division).  The forward can leave per pixel its final
// transmittance and last contributor (the state).  The backward either
// reuses the forward's sorted lists (warps taking (tile, block) items from a
// queue) or rebuilds them; it takes the last contributor and final
// transmittance from the state, or re-walks each pixel front to back for
// them, then walks back to front with the carry
// R_i = alpha_{i+1} c_{i+1} + (1 - alpha_{i+1}) R_{i+1}, recovering T_i from
// T_{i+1} / (1 - alpha_i) (alpha <= 0.99 keeps this safe), and accumulates
// d/d(x, y, z, r) per sphere as a warp sum (a six-shuffle reduce-scatter)
// and one 16-byte FP32 atomic per sphere and warp.
#include "vtx_internal.h"

namespace vtx {

cudaError_t run_binning(const Geometry &g, const Scene &sc, const Scratch &s, cudaStream_t st, StageEvents *evs,
                        bool soft);

constexpr int kSoftCap = 4096;
constexpr int kSoftNT = 256;
constexpr float kTStop = 1e-4f;
constexpr float kAMax = 0.99f;

// A tile entry as the per-pixel loop reads it from shared memory: the record's
// projection terms plus the per-sphere constants of the soft terms, computed
// once per entry when a warp stages it instead of once per pixel.
struct __align__(16) SoftPrim {
  float u0h, u0l, v0h, v0l;   // projected reference point (pixels), double-float
  float k, dz, zr, rad;       // A per pixel at zr, zr - centre depth, reference depth, radius
  float fz, inv_rad, eta, rej2;  // f / centre depth, 1 / rad, 0.05 rad, bound on rho^2 of a used sphere
  float rpx2;                 // rej2 / k^2 (px^2) when dz = 0, else +inf: the pixel-distance pre-test
  float pad[3];
};
static_assert(sizeof(SoftPrim) == 64, "SoftPrim is four 16-byte words");
static_assert(kSoftNT * sizeof(SoftPrim) >= kSoftCap * sizeof(uint16_t), "the record windows hold the sort's offsets");

constexpr size_t kSoftSmem = kSoftCap * sizeof(unsigned long long) + kSoftNT * sizeof(SoftPrim);

__device__ __forceinline__ SoftPrim soft_prim(const PrimRec &p, float f) {
  SoftPrim s;
  s.u0h = p.u0h;
  s.u0l = p.u0l;
  s.v0h = p.v0h;
  s.v0l = p.v0l;
  s.k = p.k;
  s.dz = p.dz;
  s.zr = p.zr;
  s.rad = p.rad;
  s.fz = f / (p.zr - p.dz);
  s.inv_rad = 1.0f / p.rad;
  s.eta = 0.05f * p.rad;
  // delta >= -4 px needs sqrt(rho^2) <= rad + 4 / fz; the bound is widened by
  // 0.05 % so that rounding never drops a sphere the exact test keeps.
  const float reach = p.rad + 4.0f / s.fz;
  s.rej2 = reach * reach * 1.001f + 1e-6f;
  // with dz = 0 the offset is o = k (dx, -dy, 0) and rho^2 >= |o|^2 / |u|^2 (Cauchy-Schwarz on its x, y part),
  // so d^2 > rej2 |u|^2 / k^2 (d: pixel distance to the projected centre) rejects the sphere; the 0.1 % in
  // rej2 covers the FP32 rounding of this quotient
  s.rpx2 = p.dz == 0.0f ? s.rej2 / (p.k * p.k) : __int_as_float(0x7f800000);
  s.pad[0] = s.pad[1] = s.pad[2] = 0.0f;
  return s;
}

// Per-pixel ray constants.
struct SoftPix {
  PixRay r;
  float inv_uu, inv_un;  // 1 / |u|^2, 1 / |u|
};

__device__ __forceinline__ SoftPix soft_pix(const ViewParams &v, int px, int py) {
  SoftPix x;
  x.r = pix_ray(v, px, py);
  x.inv_uu = 1.0f / x.r.uu;
  x.inv_un = 1.0f / sqrtf(x.r.uu);
  return x;
}

struct SoftTerm {
  float3 ov;        // ray origin minus centre (internal frame)
  float sst;        // ray parameter of the closest approach, relative to zr
  float rho2, rho2s, delta, sg, alpha, m, ism, si, t;
  float3 n;         // internal frame
};

// The soft term of one sphere for one pixel; false when delta < -4 px.
// nl2s = -log2(e) / sigma, so that exp(-delta / sigma) = 2^(delta nl2s).
__device__ __forceinline__ bool soft_term(const SoftPrim &p, const SoftPix &x, float nl2s, SoftTerm &o) {
  const PixRay &r = x.r;
  const float ox = __fsub_rn(__fsub_rn(r.pxc, p.u0h), p.u0l);
  const float oy = __fsub_rn(__fsub_rn(r.pyc, p.v0h), p.v0l);
  if (fmaf(ox, ox, oy * oy) > p.rpx2 * r.uu) return false;  // pixel-distance pre-test
  o.ov = make_float3(__fmul_rn(p.k, ox), __fmul_rn(-p.k, oy), p.dz);  // local_o
  const float ou = fmaf(o.ov.x, r.a, fmaf(o.ov.y, r.b, o.ov.z));
  const float oo = fmaf(o.ov.x, o.ov.x, fmaf(o.ov.y, o.ov.y, o.ov.z * o.ov.z));
  o.sst = -ou * x.inv_uu;
  o.rho2 = fmaxf(fmaf(ou, o.sst, oo), 0.0f);  // |o|^2 - (o.u)^2 / |u|^2
  if (o.rho2 > p.rej2) return false;
  o.rho2s = o.rho2 + 1e-12f;
  // hardware approximations (relative errors near 1e-7; the outputs' tolerance is 5e-5): sqrt as x rsqrt(x),
  // the sigmoid through ex2.approx and rcp.approx
  o.delta = (p.rad - o.rho2s * rsqrtf(o.rho2s)) * p.fz;
  if (!(o.delta >= -4.0f)) return false;
  o.sg = rcp_approx(1.0f + exp2_approx(o.delta * nl2s));
  o.alpha = fminf(kAMax, o.sg);
  o.m = fmaxf(fmaf(p.rad, p.rad, -o.rho2), 0.0f);
  const float m2 = fmaf(p.eta, p.eta, o.m);
  o.ism = rsqrtf(m2);
  o.si = fmaf(-(m2 * o.ism - p.eta), x.inv_un, o.sst);  // smoothed entry, relative to zr
  o.t = p.zr + o.si;
  o.n = make_float3(fmaf(o.si, r.a, o.ov.x) * p.inv_rad, fmaf(o.si, r.b, o.ov.y) * p.inv_rad,
                    (o.ov.z + o.si) * p.inv_rad);
  return true;
}

struct SoftTile {
  int img, px, py, m;
  int px0, py0;  // the tile's first column and row
  bool inside;
  uint32_t start;
  const unsigned long long *list;  // the tile's entries in (centre-depth key, id) order: shared or global memory
};

// Exact ascending order of a tile's m entries (centre-depth key << 32 | id)
// in s_e.  A one-pass counting sort first places the entries into 256 buckets
// of the tile's key range by a monotone FP32 map (every key of a bucket is <=
// every key of a later bucket, and equal keys share a bucket); each thread
// then insertion-sorts its own bucket.  A tile whose fullest bucket holds more
// than 32 entries is finished by a bitonic sort instead.  src is the list in
// global memory (read three times, L1 hits after the first); s_off (2 bytes
// per entry) is scratch.
__device__ __forceinline__ void soft_order(const unsigned long long *__restrict__ src, int m,
                                           unsigned long long *s_e, uint16_t *s_off) {
  constexpr int NB = kSoftNT;  // one bucket per thread
  __shared__ uint32_t s_cnt[NB], s_red[3], s_wt[kSoftNT / 32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  uint32_t lo = 0xffffffffu, hi = 0u;
  for (int i = threadIdx.x; i < m; i += kSoftNT) {
    const uint32_t k = (uint32_t)(src[i] >> 32);
    lo = min(lo, k);
    hi = max(hi, k);
  }
  lo = __reduce_min_sync(0xffffffffu, lo);
  hi = __reduce_max_sync(0xffffffffu, hi);
  s_cnt[threadIdx.x] = 0u;
  if (threadIdx.x == 0) {
    s_red[0] = 0xffffffffu;
    s_red[1] = 0u;
    s_red[2] = 0u;
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
  for (int i = threadIdx.x; i < m; i += kSoftNT) {
    const uint32_t k = (uint32_t)(src[i] >> 32);
    s_off[i] = (uint16_t)atomicAdd(s_cnt + min(NB - 1, (int)((float)(k - lo) * scale)), 1u);
  }
  __syncthreads();
  const uint32_t c = s_cnt[threadIdx.x];
  uint32_t inc = c;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += y;
  }
  const uint32_t cmax = __reduce_max_sync(0xffffffffu, c);
  if (lane == 31) s_wt[wid] = inc;
  if (lane == 0) atomicMax(s_red + 2, cmax);
  __syncthreads();
  uint32_t base = inc - c;
  for (int w = 0; w < wid; ++w) base += s_wt[w];
  s_cnt[threadIdx.x] = base;
  __syncthreads();
  for (int i = threadIdx.x; i < m; i += kSoftNT) {
    const unsigned long long e = src[i];
    const uint32_t k = (uint32_t)(e >> 32);
    s_e[s_cnt[min(NB - 1, (int)((float)(k - lo) * scale))] + s_off[i]] = e;
  }
  const bool small = s_red[2] <= 32u;
  __syncthreads();
  if (small) {
    for (int i = (int)base + 1; i < (int)(base + c); ++i) {
      const unsigned long long x = s_e[i];
      int j = i - 1;
      while (j >= (int)base && s_e[j] > x) {
        s_e[j + 1] = s_e[j];
        --j;
      }
      s_e[j + 1] = x;
    }
    __syncthreads();
    return;
  }
  int n2 = 1;
  while (n2 < m) n2 <<= 1;
  for (int i = m + threadIdx.x; i < n2; i += kSoftNT) s_e[i] = ~0ull;
  __syncthreads();
  for (int k = 2; k <= n2; k <<= 1) {
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int i = threadIdx.x; i < n2; i += kSoftNT) {
        const int ixj = i ^ j;
        if (ixj > i) {
          const unsigned long long a = s_e[i], b2 = s_e[ixj];
          const bool up = (i & k) == 0;
          if ((a > b2) == up) {
            s_e[i] = b2;
            s_e[ixj] = a;
          }
        }
      }
      __syncthreads();
    }
  }
}

// Ascending order of a list too long for shared memory, sorted in place in global memory by the whole CTA:
// a bitonic network written with ascending comparisons only (each stage first compares i with
// i ^ (k - 1), then i with i + j), so that padding the list to a power of two with virtual +inf entries
// never moves anything: no element is compared with a partner at or beyond m.
__device__ __noinline__ void soft_sort_global(unsigned long long *a, int m) {
  int n2 = 1;
  while (n2 < m) n2 <<= 1;
  const int half = n2 >> 1;
  for (int k = 2; k <= n2; k <<= 1) {
    const int hk = k >> 1;
    for (int t = threadIdx.x; t < half; t += blockDim.x) {
      const int i = (t / hk) * k + (t % hk);
      const int q = i ^ (k - 1);
      if (q < m) {
        const unsigned long long x = a[i], y = a[q];
        if (x > y) {
          a[i] = y;
          a[q] = x;
        }
      }
    }
    __syncthreads();
    for (int j = k >> 2; j > 0; j >>= 1) {
      for (int t = threadIdx.x; t < half; t += blockDim.x) {
        const int i = (t / j) * 2 * j + (t % j);
        const int q = i + j;
        if (q < m) {
          const unsigned long long x = a[i], y = a[q];
          if (x > y) {
            a[i] = y;
            a[q] = x;
          }
        }
      }
      __syncthreads();
    }
  }
}

// Load and order a tile's entries (shared by forward and backward).  Up to kSoftCap entries are ordered
// in shared memory; a longer list is ordered in place in the entry array, which the walk then reads.
// The forward writes the ordered list back to the entry array (store_back), so a backward call on the
// same lists loads it already ordered (presorted) instead of sorting it again.
__device__ __forceinline__ bool soft_load(const Geometry &g, long long gt, unsigned long long *entries,
                                          unsigned long long cap_entries, const uint32_t *tile_count,
                                          const uint32_t *tile_start, Status *status, unsigned long long *s_e,
                                          uint16_t *s_off, SoftTile &T, bool store_back, bool presorted) {
  T.img = (int)(gt / g.tiles_per_img);
  const int t = (int)(gt % g.tiles_per_img);
  const int tx = t % g.tiles_x, ty = t / g.tiles_x;
  T.px0 = tx * 16;
  T.py0 = ty * 16;
  // warp w covers the 8x4 block (w & 1, w >> 1) of the tile; lane l its pixel (l & 7, l >> 3)
  const int w = (int)(threadIdx.x >> 5), l = (int)(threadIdx.x & 31);
  T.px = T.px0 + 8 * (w & 1) + (l & 7);
  T.py = T.py0 + 4 * (w >> 1) + (l >> 3);
  T.inside = T.px < g.W && T.py < g.H;
  uint32_t cnt = tile_count[gt];
  T.start = tile_start[gt];
  if ((unsigned long long)T.start >= cap_entries) cnt = 0;
  else if ((unsigned long long)T.start + cnt > cap_entries) cnt = (uint32_t)(cap_entries - T.start);
  if (threadIdx.x == 0) atomicMax(&status->max_list, cnt);
  T.m = (int)cnt;
  T.list = s_e;
  if (cnt == 0) return false;
  if (cnt > (uint32_t)kSoftCap) {
    if (!presorted) soft_sort_global(entries + T.start, T.m);
    T.list = entries + T.start;
  } else if (presorted) {
    for (int i = threadIdx.x; i < T.m; i += kSoftNT) s_e[i] = entries[T.start + i];
    __syncthreads();
  } else {
    soft_order(entries + T.start, T.m, s_e, s_off);
    if (store_back)
      for (int i = threadIdx.x; i < T.m; i += kSoftNT) entries[T.start + i] = s_e[i];
  }
  return true;
}

// Each warp walks the sorted list on its own (no block barrier after the
// sort, so a warp of saturated pixels never waits for a warp of silhouette
// pixels): it stages 32 entries at a time, lane i converting entry c0 + i, in
// its private 32-slot window of shared memory.
//
// Staging also culls the window for the warp.  The warp covers an 8x4 pixel
// block (lane l at column l & 7, row l >> 3); `am` marks the lanes still
// compositing.  For a sphere whose reference
// point is its centre (dz = 0) the offset at the reference depth is
// o = k (du, -dv, 0) with (du, dv) the pixel offset from the projected centre,
// and rho^2 = |o|^2 - (o.u)^2 / |u|^2 >= |o|^2 / |u|^2 (Cauchy-Schwarz on the
// x, y part), so rho^2 > rej2 whenever k^2 d^2 > rej2 |u|^2_max.  Entries whose
// disc of that radius misses the bounding rectangle of the active lanes'
// pixel centres are dropped from the returned mask; the radius is widened
// (0.01 % plus 1e-3 px plus 2e-7 of the coordinates) to cover FP32 rounding.
// The record index of entry j of the tile's list (0 past its end); loaded one window ahead of its use.
__device__ __forceinline__ uint32_t soft_rec_index(const Geometry &g, const uint32_t *__restrict__ rec_of,
                                                   const SoftTile &T, int j) {
  return (j >= 0 && j < T.m) ? rec_of[(long long)T.img * g.n_atoms + (uint32_t)T.list[j]] : 0u;
}

__device__ __forceinline__ unsigned soft_stage(const PrimRec *__restrict__ recs, uint32_t ridx, const SoftTile &T,
                                               int c0, float f, SoftPrim *s_w, unsigned am, float col0, float row0,
                                               float uu_max) {
  const int lane = threadIdx.x & 31;
  const int j = c0 + lane;
  bool keep = false;
  if (j < T.m) {
    const SoftPrim sp = soft_prim(recs[ridx], f);
    s_w[lane] = sp;
    const unsigned cols = (am | (am >> 8) | (am >> 16) | (am >> 24)) & 0xffu;
    const unsigned rows = ((am & 0xffu) ? 1u : 0u) | ((am & 0xff00u) ? 2u : 0u) | ((am & 0xff0000u) ? 4u : 0u) |
                          ((am & 0xff000000u) ? 8u : 0u);
    const float rx0 = col0 + (float)(__ffs(cols) - 1), rx1 = col0 + (float)(31 - __clz(cols));
    const float ry0 = row0 + (float)(__ffs(rows) - 1), ry1 = row0 + (float)(31 - __clz(rows));
    const float cu = sp.u0h + sp.u0l, cv = sp.v0h + sp.v0l;
    const float dx = fmaxf(fmaxf(rx0 - cu, cu - rx1), 0.0f);
    const float dy = fmaxf(fmaxf(ry0 - cv, cv - ry1), 0.0f);
    const float r2 = sp.rej2 * uu_max;  // approximate root and quotient: the 0.01 % widening covers their error
    const float rt = __fdividef(r2 * rsqrtf(r2), sp.k) * 1.0001f + 1e-3f + 2e-7f * (fabsf(cu) + fabsf(cv));
    keep = sp.dz != 0.0f || !(dx * dx + dy * dy > rt * rt);
  }
  return __ballot_sync(0xffffffffu, keep);
}

// state (optional, [n_img][H][W]): per pixel the final transmittance (float
// bits) and 1 + the sorted-list position of its last contributor (0: none),
// which lets the backward pass start its back-to-front walk directly.
#ifndef VTX_SOFT_FWD_MINB
#define VTX_SOFT_FWD_MINB 4
#endif
// One tile of the forward pass (called by every thread of the CTA).
__device__ __forceinline__ void soft_fwd_tile(const Geometry &g, long long gt, const PrimRec *__restrict__ recs,
                                              const uint32_t *__restrict__ rec_of, unsigned long long *entries,
                                              unsigned long long cap_entries, const uint32_t *__restrict__ tile_count,
                                              const uint32_t *__restrict__ tile_start, Status *status, float *cov,
                                              float *dep, float *nrm, uint2 *state, unsigned long long *s_e,
                                              SoftPrim *s_w) {
  SoftTile T;
  const bool any = soft_load(g, gt, entries, cap_entries, tile_count, tile_start, status, s_e,
                             reinterpret_cast<uint16_t *>(s_w - (threadIdx.x & ~31)), T, true, false);
  const ViewParams &v = g.views[T.img % g.n_views];
  const SoftPix x = soft_pix(v, T.px, T.py);
  const float inv_sigma = 1.0f / g.sigma;
  const float nl2s = -1.4426950408889634f * inv_sigma;  // exp(-delta / sigma) = 2^(delta nl2s)
  const float uu_max = __uint_as_float(__reduce_max_sync(0xffffffffu, __float_as_uint(x.r.uu)));
  const float col0 = (float)(T.px0 + 8 * (int)((threadIdx.x >> 5) & 1)) + 0.5f;
  const float row0 = (float)(T.py0 + 4 * (int)(threadIdx.x >> 6)) + 0.5f;
  const int lane = threadIdx.x & 31;
  float A = 0.0f, D = 0.0f, N0 = 0.0f, N1 = 0.0f, N2 = 0.0f, Tr = 1.0f;
  int last = -1;
  unsigned used = 0u;
  bool done = !T.inside;
  if (any) {
    uint32_t ridx = soft_rec_index(g, rec_of, T, lane);
    for (int c0 = 0; c0 < T.m; c0 += 32) {
      const unsigned am = __ballot_sync(0xffffffffu, !done);
      if (am == 0u) break;
      const uint32_t next = soft_rec_index(g, rec_of, T, c0 + 32 + lane);  // the next window's, in flight now
      const unsigned keep = soft_stage(recs, ridx, T, c0, v.f, s_w, am, col0, row0, uu_max);
      ridx = next;
      __syncwarp();
      for (unsigned b = keep; b != 0u; b &= b - 1u) {
        if (done) continue;
        const int q = __ffs(b) - 1;
        SoftTerm o;
        if (!soft_term(s_w[q], x, nl2s, o)) continue;
        const float w = o.alpha * Tr;
        A += w;
        D = fmaf(w, o.t, D);
        N0 = fmaf(w, o.n.x, N0);
        N1 = fmaf(w, o.n.y, N1);
        N2 = fmaf(-w, o.n.z, N2);
        Tr *= 1.0f - o.alpha;
        last = c0 + q;
        ++used;
        if (Tr < kTStop) done = true;
      }
      __syncwarp();
    }
  }
  // composited terms, one atomic per warp (the algorithmic work of the pass)
  const unsigned wused = __reduce_add_sync(0xffffffffu, used);
  if (lane == 0 && wused) atomicAdd(&status->n_terms, (unsigned long long)wused);
  if (T.inside) {
    if (state)
      state[(long long)T.img * g.pix_per_img + (long long)T.py * g.W + T.px] =
          make_uint2(__float_as_uint(Tr), (uint32_t)(last + 1));
    const long long ppi = g.pix_per_img;
    const long long p = (long long)T.py * g.W + T.px;
    cov[(long long)T.img * ppi + p] = A;
    dep[(long long)T.img * ppi + p] = D;
    float *nb = nrm + (long long)T.img * 3 * ppi + p;
    nb[0] = N0;
    nb[ppi] = N1;
    nb[2 * ppi] = N2;
  }
}

// Forward: one CTA per tile, the empty ones writing their zeros (overlapped with the busy tiles).
// state (optional, [n_img][H][W]): per pixel the final transmittance (float
// bits) and 1 + the sorted-list position of its last contributor (0: none),
// which lets the backward pass start its back-to-front walk directly.
__global__ __launch_bounds__(kSoftNT, VTX_SOFT_FWD_MINB) void k_soft_fwd(Geometry g, const PrimRec *__restrict__ recs,
                                                      const uint32_t *__restrict__ rec_of,
                                                      unsigned long long *entries,
                                                      unsigned long long cap_entries,
                                                      const uint32_t *__restrict__ tile_count,
                                                      const uint32_t *__restrict__ tile_start,
                                                      const uint32_t *__restrict__ tile_list, Status *status,
                                                      float *cov, float *dep, float *nrm, uint2 *state) {
  extern __shared__ __align__(16) unsigned char smem[];
  unsigned long long *s_e = reinterpret_cast<unsigned long long *>(smem);
  SoftPrim *s_w = reinterpret_cast<SoftPrim *>(smem + kSoftCap * sizeof(unsigned long long)) + (threadIdx.x & ~31);
  // every tile, longest list first when the scan listed them all (empty tiles last), else in index order
  const long long gt = tile_list ? (long long)tile_list[blockIdx.x] : (long long)blockIdx.x;
  soft_fwd_tile(g, gt, recs, rec_of, entries, cap_entries, tile_count, tile_start, status, cov, dep, nrm, state, s_e,
                s_w);
}

// Sum of four per-lane values over the warp, scattered: lanes 0, 8, 16 and 24
// receive the sums of a0, a1, a2 and a3 (six shuffles instead of twenty).
__device__ __forceinline__ float warp_sum4_scatter(float a0, float a1, float a2, float a3, int lane) {
  const bool hi16 = (lane & 16) != 0;
  float k0 = hi16 ? a2 : a0, k1 = hi16 ? a3 : a1;
  const float s0 = hi16 ? a0 : a2, s1 = hi16 ? a1 : a3;
  k0 += __shfl_xor_sync(0xffffffffu, s0, 16);
  k1 += __shfl_xor_sync(0xffffffffu, s1, 16);
  const bool hi8 = (lane & 8) != 0;
  float k = hi8 ? k1 : k0;
  k += __shfl_xor_sync(0xffffffffu, hi8 ? k0 : k1, 8);
  k += __shfl_xor_sync(0xffffffffu, k, 4);
  k += __shfl_xor_sync(0xffffffffu, k, 2);
  k += __shfl_xor_sync(0xffffffffu, k, 1);
  return k;
}

// One tile of the backward pass (called by every thread of the CTA).
__device__ __forceinline__ void soft_bwd_tile(const Geometry &g, long long gt, const PrimRec *__restrict__ recs,
                                              const uint32_t *__restrict__ rec_of, unsigned long long *entries,
                                              unsigned long long cap_entries, const uint32_t *__restrict__ tile_count,
                                              const uint32_t *__restrict__ tile_start, Status *status,
                                              const float *gcov, const float *gdep, const float *gnrm,
                                              const uint2 *__restrict__ state, float *grad, unsigned long long *s_e,
                                              SoftPrim *s_w, bool presorted);

// The backward of one warp: its 8x4 pixel block wblk of tile T, whose sorted list T.list is in shared or
// global memory; s_w is the warp's 32-entry window.
__device__ __forceinline__ void soft_bwd_walk(const Geometry &g, const SoftTile &T, int wblk,
                                              const PrimRec *__restrict__ recs, const uint32_t *__restrict__ rec_of,
                                              const float *gcov, const float *gdep, const float *gnrm,
                                              const uint2 *__restrict__ state, float *grad, SoftPrim *s_w) {
  const ViewParams &v = g.views[T.img % g.n_views];
  const SoftPix x = soft_pix(v, T.px, T.py);
  const PixRay &r = x.r;
  const float inv_sigma = 1.0f / g.sigma;
  const float nl2s = -1.4426950408889634f * inv_sigma;
  const long long ppi = g.pix_per_img;
  const long long p = (long long)T.py * g.W + T.px;
  float gA = 0.0f, gD = 0.0f;
  float3 gN = make_float3(0.0f, 0.0f, 0.0f);
  if (T.inside) {
    const long long q = (long long)T.img * ppi + p;
    if (gcov) gA = gcov[q];
    if (gdep) gD = gdep[q];
    if (gnrm) {
      const float *b = gnrm + (long long)T.img * 3 * ppi + p;
      gN = make_float3(b[0], b[ppi], -b[2 * ppi]);  // to the internal frame
    }
  }
  const bool need = T.inside && (gA != 0.0f || gD != 0.0f || gN.x != 0.0f || gN.y != 0.0f || gN.z != 0.0f);
  // pass 1: front to back, last contributor and final transmittance (read from the forward call's state
  // when it left one)
  const float uu_max = __uint_as_float(__reduce_max_sync(0xffffffffu, __float_as_uint(r.uu)));
  const float col0 = (float)(T.px0 + 8 * (wblk & 1)) + 0.5f;
  const float row0 = (float)(T.py0 + 4 * (wblk >> 1)) + 0.5f;
  float Tr = 1.0f;
  int last = -1;
  bool done = !need;
  if (state) {
    if (need) {
      const uint2 sv = state[(long long)T.img * ppi + p];
      Tr = __uint_as_float(sv.x);
      last = min((int)sv.y - 1, T.m - 1);
    }
    done = true;
  }
  const int lane = threadIdx.x & 31;
  uint32_t ridx = soft_rec_index(g, rec_of, T, lane);  // lane stages entry c0 + lane for the whole warp
  for (int c0 = 0; c0 < T.m && !__all_sync(0xffffffffu, done); c0 += 32) {
    const unsigned am = __ballot_sync(0xffffffffu, !done);
    if (am == 0u) break;
    const uint32_t next = soft_rec_index(g, rec_of, T, c0 + 32 + lane);
    const unsigned keep = soft_stage(recs, ridx, T, c0, v.f, s_w, am, col0, row0, uu_max);
    ridx = next;
    __syncwarp();
    for (unsigned b = keep; b != 0u; b &= b - 1u) {
      if (done) continue;
      const int q = __ffs(b) - 1;
      SoftTerm o;
      if (!soft_term(s_w[q], x, nl2s, o)) continue;
      Tr *= 1.0f - o.alpha;
      last = c0 + q;
      if (Tr < kTStop) done = true;
    }
    __syncwarp();
  }
  const int wlast = __reduce_max_sync(0xffffffffu, last);
  if (wlast < 0) return;
  // pass 2: back to front; per-sphere sums leave the warp as one 16-byte atomic
  const float ugn0 = fmaf(r.a, gN.x, fmaf(r.b, gN.y, gN.z));
  float R = 0.0f, Tc = Tr;
  ridx = soft_rec_index(g, rec_of, T, (wlast / 32) * 32 + lane);
  for (int c0 = (wlast / 32) * 32; c0 >= 0; c0 -= 32) {
    const unsigned am = __ballot_sync(0xffffffffu, last >= c0);
    const uint32_t prev = soft_rec_index(g, rec_of, T, c0 - 32 + lane);  // the previous window's, in flight now
    if (am == 0u) {
      ridx = prev;
      continue;
    }
    __syncwarp();
    unsigned keep = soft_stage(recs, ridx, T, c0, v.f, s_w, am, col0, row0, uu_max);
    ridx = prev;
    if (wlast - c0 < 31) keep &= (2u << (wlast - c0)) - 1u;
    __syncwarp();
    while (keep != 0u) {
      const int q = 31 - __clz(keep);
      keep &= ~(1u << q);
      const SoftPrim &pr = s_w[q];
      float gx = 0.0f, gy = 0.0f, gz = 0.0f, grr = 0.0f;
      SoftTerm o;
      if (c0 + q <= last && soft_term(pr, x, nl2s, o)) {
        const float Ti = Tc / (1.0f - o.alpha);
        const float w = o.alpha * Ti;
        const float ci = gA + gD * o.t + gN.x * o.n.x + gN.y * o.n.y + gN.z * o.n.z;
        const float dalpha = Ti * (ci - R);
        R = o.alpha * ci + (1.0f - o.alpha) * R;
        Tc = Ti;
        const float dadd = o.sg < kAMax ? o.sg * (1.0f - o.sg) * inv_sigma : 0.0f;
        const float dd = dalpha * dadd;
        // closest-approach offset q = C - (o + s u), |q|^2 = rho^2
        const float3 qv = make_float3(-fmaf(o.sst, r.a, o.ov.x), -fmaf(o.sst, r.b, o.ov.y), -(o.ov.z + o.sst));
        const float ddf = dd * pr.fz;
        const float isq = rsqrtf(o.rho2s);
        // delta(C, r)
        gx = -ddf * qv.x * isq;
        gy = -ddf * qv.y * isq;
        gz = -ddf * qv.z * isq - ddf * o.delta * v.inv_f;  // d delta / d zc = -delta / zc = -delta fz / f
        grr = ddf;
        // t_i(C, r) and n_i = (t_i u - C) / r
        float c2 = 0.0f, dg_dr = 0.0f;
        if (o.m > 0.0f) {
          c2 = -o.ism * x.inv_un;                       // 2 (dg / drho^2) / |u|
          dg_dr = fmaf(0.05f, pr.eta, pr.rad) * o.ism - 0.05f;
        }
        const float dtx = fmaf(r.a, x.inv_uu, -c2 * qv.x);
        const float dty = fmaf(r.b, x.inv_uu, -c2 * qv.y);
        const float dtz = x.inv_uu - c2 * qv.z;
        const float dtr = -dg_dr * x.inv_un;
        const float ut = w * gD;
        const float ugn = w * ugn0;
        const float inv = pr.inv_rad;
        gx += ut * dtx + (dtx * ugn - w * gN.x) * inv;
        gy += ut * dty + (dty * ugn - w * gN.y) * inv;
        gz += ut * dtz + (dtz * ugn - w * gN.z) * inv;
        grr += ut * dtr + (ugn * dtr - w * (gN.x * o.n.x + gN.y * o.n.y + gN.z * o.n.z)) * inv;
      }
      const bool nz = gx != 0.0f || gy != 0.0f || gz != 0.0f || grr != 0.0f;
      if (__any_sync(0xffffffffu, nz)) {
        const float sum = warp_sum4_scatter(gx, gy, gz, grr, lane);
        const float sy = __shfl_sync(0xffffffffu, sum, 8);
        const float sz = __shfl_sync(0xffffffffu, sum, 16);
        const float sr = __shfl_sync(0xffffffffu, sum, 24);
        if (lane == 0) {
          const uint32_t id = (uint32_t)T.list[c0 + q];
          const float4 wv = make_float4(v.R[0] * sum + v.U[0] * sy + v.F[0] * sz,
                                        v.R[1] * sum + v.U[1] * sy + v.F[1] * sz,
                                        v.R[2] * sum + v.U[2] * sy + v.F[2] * sz, sr);
          atomicAdd(reinterpret_cast<float4 *>(grad) + id, wv);
        }
      }
    }
  }
}

__device__ __forceinline__ void soft_bwd_tile(const Geometry &g, long long gt, const PrimRec *__restrict__ recs,
                                              const uint32_t *__restrict__ rec_of, unsigned long long *entries,
                                              unsigned long long cap_entries, const uint32_t *__restrict__ tile_count,
                                              const uint32_t *__restrict__ tile_start, Status *status,
                                              const float *gcov, const float *gdep, const float *gnrm,
                                              const uint2 *__restrict__ state, float *grad, unsigned long long *s_e,
                                              SoftPrim *s_w, bool presorted) {
  SoftTile T;
  if (!soft_load(g, gt, entries, cap_entries, tile_count, tile_start, status, s_e,
                 reinterpret_cast<uint16_t *>(s_w - (threadIdx.x & ~31)), T, false, presorted))
    return;
  soft_bwd_walk(g, T, (int)(threadIdx.x >> 5), recs, rec_of, gcov, gdep, gnrm, state, grad, s_w);
}

// Persistent backward over the non-empty tiles (as the forward).
__global__ __launch_bounds__(kSoftNT) void k_soft_bwd(Geometry g, const PrimRec *__restrict__ recs,
                                                      const uint32_t *__restrict__ rec_of,
                                                      unsigned long long *entries,
                                                      unsigned long long cap_entries,
                                                      const uint32_t *__restrict__ tile_count,
                                                      const uint32_t *__restrict__ tile_start,
                                                      const uint32_t *__restrict__ tile_list, Status *status,
                                                      const float *gcov, const float *gdep, const float *gnrm,
                                                      const uint2 *__restrict__ state, float *grad, int presorted) {
  extern __shared__ __align__(16) unsigned char smem[];
  unsigned long long *s_e = reinterpret_cast<unsigned long long *>(smem);
  SoftPrim *s_w = reinterpret_cast<SoftPrim *>(smem + kSoftCap * sizeof(unsigned long long)) + (threadIdx.x & ~31);
  __shared__ uint32_t s_li;
  const uint32_t n_list = status->n_list;
  for (;;) {
    if (threadIdx.x == 0) s_li = atomicAdd(&status->soft_next, 1u);
    __syncthreads();
    const uint32_t li = s_li;
    if (li >= n_list) break;
    soft_bwd_tile(g, tile_list[li], recs, rec_of, entries, cap_entries, tile_count, tile_start, status, gcov, gdep,
                  gnrm, state, grad, s_e, s_w, presorted != 0);
    __syncthreads();
  }
}

// Backward on the forward call's lists, already sorted in the entry array: each warp takes (tile, 8x4 block)
// items from a queue -- the non-empty tiles longest first, eight blocks each -- and walks the tile's list in
// global memory on its own.  No step needs the whole tile, so there is no block barrier: a warp that finishes
// its block early takes the next item instead of waiting for the tile's slowest warp.
__global__ __launch_bounds__(kSoftNT, 4) void k_soft_bwd_warps(Geometry g, const PrimRec *__restrict__ recs,
                                                            const uint32_t *__restrict__ rec_of,
                                                            const unsigned long long *__restrict__ entries,
                                                            unsigned long long cap_entries,
                                                            const uint32_t *__restrict__ tile_count,
                                                            const uint32_t *__restrict__ tile_start,
                                                            const uint32_t *__restrict__ tile_list, Status *status,
                                                            const float *gcov, const float *gdep, const float *gnrm,
                                                            const uint2 *__restrict__ state, float *grad) {
  __shared__ SoftPrim s_win[kSoftNT];  // a 32-entry window per warp
  SoftPrim *s_w = s_win + (threadIdx.x & ~31);
  const int lane = threadIdx.x & 31;
  const uint32_t n_items = status->n_list * 8u;
  for (;;) {
    uint32_t item = 0u;
    if (lane == 0) item = atomicAdd(&status->soft_next, 1u);
    item = __shfl_sync(0xffffffffu, item, 0);
    if (item >= n_items) break;
    const long long gt = tile_list[item >> 3];
    const int wblk = (int)(item & 7u);
    SoftTile T;
    T.img = (int)(gt / g.tiles_per_img);
    const int t = (int)(gt % g.tiles_per_img);
    T.px0 = (t % g.tiles_x) * 16;
    T.py0 = (t / g.tiles_x) * 16;
    T.px = T.px0 + 8 * (wblk & 1) + (lane & 7);
    T.py = T.py0 + 4 * (wblk >> 1) + (lane >> 3);
    T.inside = T.px < g.W && T.py < g.H;
    uint32_t cnt = tile_count[gt];
    T.start = tile_start[gt];
    if ((unsigned long long)T.start >= cap_entries) cnt = 0;
    else if ((unsigned long long)T.start + cnt > cap_entries) cnt = (uint32_t)(cap_entries - T.start);
    T.m = (int)cnt;
    T.list = entries + T.start;
    if (cnt > 0) soft_bwd_walk(g, T, wblk, recs, rec_of, gcov, gdep, gnrm, state, grad, s_w);
    __syncwarp();
  }
}

cudaError_t run_soft_pipeline(const Geometry &g, const Scene &sc, const Scratch &s, float *cov, float *depth,
                              float *normal, const float *g_cov, const float *g_depth, const float *g_normal,
                              float *grad, uint2 *state, bool reuse_lists, cudaStream_t st, StageEvents *evs) {
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_soft_fwd, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSoftSmem);
    cudaFuncSetAttribute(k_soft_bwd, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSoftSmem);
    attr = true;
  }
  const bool reuse = reuse_lists && grad != nullptr;
  if (reuse) {
    // the lists, records and tile order of the forward call are still in place; only the backward's tile
    // queue counter (which the forward leaves untouched) is reset
    cudaMemsetAsync(&s.status->soft_next, 0, sizeof(s.status->soft_next), st);
  } else {
    cudaError_t e = run_binning(g, sc, s, st, evs, true);
    if (e != cudaSuccess) return e;
  }
  const long long n_tiles = (long long)g.n_img * g.tiles_per_img;
  // persistent backward CTAs: as many as fit at once (4 per SM), never more than there are tiles
  const long long most = 4LL * sm_count();
  const unsigned grid = (unsigned)(n_tiles < most ? (n_tiles > 0 ? n_tiles : 1) : most);
  if (grad == nullptr) {
    k_soft_fwd<<<(unsigned)n_tiles, kSoftNT, kSoftSmem, st>>>(g, s.recs, s.rec_of, s.entries, s.cap_entries,
                                                             s.tile_count, s.tile_start,
                                                             n_tiles <= kScanSingleMax ? s.tile_list : nullptr,
                                                             s.status, cov, depth, normal, state);
  } else {
    cudaMemsetAsync(grad, 0, sizeof(float) * 4 * (size_t)g.n_atoms, st);
    if (reuse)
      k_soft_bwd_warps<<<(unsigned)most, kSoftNT, 0, st>>>(g, s.recs, s.rec_of, s.entries, s.cap_entries,
                                                           s.tile_count, s.tile_start, s.tile_list, s.status, g_cov,
                                                           g_depth, g_normal, state, grad);
    else
      k_soft_bwd<<<grid, kSoftNT, kSoftSmem, st>>>(g, s.recs, s.rec_of, s.entries, s.cap_entries, s.tile_count,
                                                   s.tile_start, s.tile_list, s.status, g_cov, g_depth, g_normal,
                                                   state, grad, 0);
  }
  if (evs && evs->ev && evs->n > 5) cudaEventRecord(evs->ev[5], st);
  if (evs && evs->ev && evs->n > 6) cudaEventRecord(evs->ev[6], st);
  if (evs && evs->ev && evs->n > 7) cudaEventRecord(evs->ev[7], st);
  return cudaGetLastError();
}

}  // namespace vtx
