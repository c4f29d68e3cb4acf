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
// is shared with the hard-edge path; each tile CTA sorts its list by
// (centre depth key, id) in shared memory.  The backward kernel rebuilds the
// lists, re-walks each pixel front to back to find its last contributor and
// final transmittance, then walks back to front with the carry
// R_i = alpha_{i+1} c_{i+1} + (1 - alpha_{i+1}) R_{i+1}, recovering T_i from
// T_{i+1} / (1 - alpha_i) (alpha <= 0.99 keeps this safe), and accumulates
// d/d(x, y, z, r) per sphere with warp reductions and FP32 atomics.
#include "vtx_internal.h"

namespace vtx {

cudaError_t run_binning(const Geometry &g, const Scene &sc, const Scratch &s, cudaStream_t st, StageEvents *evs,
                        bool soft);

constexpr int kSoftCap = 4096;
constexpr int kSoftNT = 256;
constexpr float kTStop = 1e-4f;
constexpr float kAMax = 0.99f;
constexpr size_t kSoftSmem = kSoftCap * sizeof(unsigned long long) + kSoftNT * sizeof(PrimRec);

struct SoftTerm {
  float alpha, sg, t, delta;
  float3 n;      // internal frame
  float3 q;      // centre minus closest ray point (internal frame)
  float sq, sm, m, zc, rho2;
};

__device__ __forceinline__ bool soft_term(const PrimRec &p, const PixRay &r, float f, float sigma, SoftTerm &o) {
  float3 ov = local_o(p.u0h, p.u0l, p.v0h, p.v0l, p.k, p.dz, r);
  float ou = fmaf(ov.x, r.a, fmaf(ov.y, r.b, ov.z));
  float oo = fmaf(ov.x, ov.x, fmaf(ov.y, ov.y, ov.z * ov.z));
  float sst = -ou / r.uu;
  o.rho2 = fmaxf(oo - ou * ou / r.uu, 0.0f);
  o.zc = p.zr - p.dz;
  o.sq = sqrtf(o.rho2 + 1e-12f);
  o.delta = (p.rad - o.sq) * f / o.zc;
  if (!(o.delta >= -4.0f)) return false;
  o.sg = 1.0f / (1.0f + expf(-o.delta / sigma));
  o.alpha = fminf(kAMax, o.sg);
  float eta = 0.05f * p.rad;
  o.m = fmaxf(p.rad * p.rad - o.rho2, 0.0f);
  o.sm = sqrtf(o.m + eta * eta);
  float gv = o.sm - eta;
  float si = sst - gv / sqrtf(r.uu);
  o.t = p.zr + si;
  float inv = 1.0f / p.rad;
  o.n = make_float3((ov.x + si * r.a) * inv, (ov.y + si * r.b) * inv, (ov.z + si) * inv);
  o.q = make_float3(-(ov.x + sst * r.a), -(ov.y + sst * r.b), -(ov.z + sst));
  return true;
}

struct SoftTile {
  int img, px, py, m;
  bool inside;
  uint32_t start;
};

// Load and sort a tile's entries (shared by forward and backward).
__device__ __forceinline__ bool soft_load(const Geometry &g, const unsigned long long *entries,
                                          unsigned long long cap_entries, const uint32_t *tile_count,
                                          const uint32_t *tile_start, Status *status, unsigned long long *s_e,
                                          SoftTile &T) {
  const long long gt = blockIdx.x;
  T.img = (int)(gt / g.tiles_per_img);
  const int t = (int)(gt % g.tiles_per_img);
  const int tx = t % g.tiles_x, ty = t / g.tiles_x;
  T.px = tx * 16 + (threadIdx.x & 15);
  T.py = ty * 16 + (threadIdx.x >> 4);
  T.inside = T.px < g.W && T.py < g.H;
  uint32_t cnt = tile_count[gt];
  T.start = tile_start[gt];
  if ((unsigned long long)T.start >= cap_entries) cnt = 0;
  else if ((unsigned long long)T.start + cnt > cap_entries) cnt = (uint32_t)(cap_entries - T.start);
  if (cnt > (uint32_t)kSoftCap) {
    if (threadIdx.x == 0) atomicOr(&status->overflow, 8u);
    cnt = kSoftCap;
  }
  if (threadIdx.x == 0) atomicMax(&status->max_list, cnt);
  T.m = (int)cnt;
  if (cnt == 0) return false;
  int n2 = 1;
  while (n2 < T.m) n2 <<= 1;
  for (int i = threadIdx.x; i < n2; i += kSoftNT) s_e[i] = i < T.m ? entries[T.start + i] : ~0ull;
  __syncthreads();
  for (int k = 2; k <= n2; k <<= 1) {
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int i = threadIdx.x; i < n2; i += kSoftNT) {
        int ixj = i ^ j;
        if (ixj > i) {
          unsigned long long a = s_e[i], b = s_e[ixj];
          bool up = (i & k) == 0;
          if ((a > b) == up) {
            s_e[i] = b;
            s_e[ixj] = a;
          }
        }
      }
      __syncthreads();
    }
  }
  return true;
}

__global__ __launch_bounds__(kSoftNT) void k_soft_fwd(Geometry g, const PrimRec *__restrict__ recs,
                                                      const uint32_t *__restrict__ rec_of,
                                                      const unsigned long long *__restrict__ entries,
                                                      unsigned long long cap_entries,
                                                      const uint32_t *__restrict__ tile_count,
                                                      const uint32_t *__restrict__ tile_start, Status *status,
                                                      float *cov, float *dep, float *nrm) {
  extern __shared__ __align__(16) unsigned char smem[];
  unsigned long long *s_e = reinterpret_cast<unsigned long long *>(smem);
  PrimRec *s_r = reinterpret_cast<PrimRec *>(smem + kSoftCap * sizeof(unsigned long long));
  SoftTile T;
  const bool any = soft_load(g, entries, cap_entries, tile_count, tile_start, status, s_e, T);
  const ViewParams &v = g.views[T.img % g.n_views];
  const PixRay r = pix_ray(v, T.px, T.py);
  float A = 0.0f, D = 0.0f, N0 = 0.0f, N1 = 0.0f, N2 = 0.0f, Tr = 1.0f;
  bool done = !T.inside;
  if (any) {
    for (int c0 = 0; c0 < T.m; c0 += kSoftNT) {
      if (__syncthreads_and(done)) break;
      const int j = c0 + threadIdx.x;
      if (j < T.m) s_r[threadIdx.x] = recs[rec_of[(long long)T.img * g.n_atoms + (uint32_t)s_e[j]]];
      __syncthreads();
      const int nj = min(kSoftNT, T.m - c0);
      for (int q = 0; q < nj && !done; ++q) {
        SoftTerm o;
        if (!soft_term(s_r[q], r, v.f, g.sigma, o)) continue;
        float w = o.alpha * Tr;
        A += w;
        D += w * o.t;
        N0 += w * o.n.x;
        N1 += w * o.n.y;
        N2 -= w * o.n.z;
        Tr *= 1.0f - o.alpha;
        if (Tr < kTStop) done = true;
      }
      __syncthreads();
    }
  }
  if (T.inside) {
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

__global__ __launch_bounds__(kSoftNT) void k_soft_bwd(Geometry g, const PrimRec *__restrict__ recs,
                                                      const uint32_t *__restrict__ rec_of,
                                                      const unsigned long long *__restrict__ entries,
                                                      unsigned long long cap_entries,
                                                      const uint32_t *__restrict__ tile_count,
                                                      const uint32_t *__restrict__ tile_start, Status *status,
                                                      const float *gcov, const float *gdep, const float *gnrm,
                                                      float *grad) {
  extern __shared__ __align__(16) unsigned char smem[];
  unsigned long long *s_e = reinterpret_cast<unsigned long long *>(smem);
  PrimRec *s_r = reinterpret_cast<PrimRec *>(smem + kSoftCap * sizeof(unsigned long long));
  __shared__ int s_maxlast;
  SoftTile T;
  if (!soft_load(g, entries, cap_entries, tile_count, tile_start, status, s_e, T)) return;
  const ViewParams &v = g.views[T.img % g.n_views];
  const PixRay r = pix_ray(v, T.px, T.py);
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
  // pass 1: front to back, last contributor and final transmittance
  float Tr = 1.0f;
  int last = -1;
  bool done = !need;
  if (threadIdx.x == 0) s_maxlast = -1;
  for (int c0 = 0; c0 < T.m; c0 += kSoftNT) {
    if (__syncthreads_and(done)) break;
    const int j = c0 + threadIdx.x;
    if (j < T.m) s_r[threadIdx.x] = recs[rec_of[(long long)T.img * g.n_atoms + (uint32_t)s_e[j]]];
    __syncthreads();
    const int nj = min(kSoftNT, T.m - c0);
    for (int q = 0; q < nj && !done; ++q) {
      SoftTerm o;
      if (!soft_term(s_r[q], r, v.f, g.sigma, o)) continue;
      Tr *= 1.0f - o.alpha;
      last = c0 + q;
      if (Tr < kTStop) done = true;
    }
    __syncthreads();
  }
  if (last >= 0) atomicMax(&s_maxlast, last);
  __syncthreads();
  const int maxlast = s_maxlast;
  if (maxlast < 0) return;
  // pass 2: back to front
  const int lane = threadIdx.x & 31;
  const float f = v.f;
  const float un = sqrtf(r.uu);
  float R = 0.0f, Tc = Tr;
  for (int c0 = (maxlast / kSoftNT) * kSoftNT; c0 >= 0; c0 -= kSoftNT) {
    __syncthreads();
    const int j = c0 + threadIdx.x;
    if (j < T.m) s_r[threadIdx.x] = recs[rec_of[(long long)T.img * g.n_atoms + (uint32_t)s_e[j]]];
    __syncthreads();
    const int nj = min(kSoftNT, T.m - c0);
    for (int q = nj - 1; q >= 0; --q) {
      const PrimRec &pr = s_r[q];
      float gx = 0.0f, gy = 0.0f, gz = 0.0f, grr = 0.0f;
      SoftTerm o;
      if (need && c0 + q <= last && soft_term(pr, r, f, g.sigma, o)) {
        const float Ti = Tc / (1.0f - o.alpha);
        const float w = o.alpha * Ti;
        const float ci = gA + gD * o.t + gN.x * o.n.x + gN.y * o.n.y + gN.z * o.n.z;
        const float dalpha = Ti * (ci - R);
        R = o.alpha * ci + (1.0f - o.alpha) * R;
        Tc = Ti;
        const float rad = pr.rad;
        const float dadd = o.sg < kAMax ? o.sg * (1.0f - o.sg) / g.sigma : 0.0f;
        const float dd = dalpha * dadd;
        const float fz = f / o.zc;
        // delta(C, r)
        gx = -dd * fz * o.q.x / o.sq;
        gy = -dd * fz * o.q.y / o.sq;
        gz = -dd * fz * o.q.z / o.sq - dd * o.delta / o.zc;
        grr = dd * fz;
        // t_i(C, r) and n_i = (t_i u - C) / r
        float dg_drho2 = 0.0f, dg_dr = 0.0f;
        if (o.m > 0.0f) {
          const float eta = 0.05f * rad;
          dg_drho2 = -0.5f / o.sm;
          dg_dr = (rad + 0.05f * eta) / o.sm - 0.05f;
        }
        const float c2 = 2.0f * dg_drho2 / un;
        const float dtx = r.a / r.uu - c2 * o.q.x;
        const float dty = r.b / r.uu - c2 * o.q.y;
        const float dtz = 1.0f / r.uu - c2 * o.q.z;
        const float dtr = -dg_dr / un;
        const float ut = w * gD;
        const float ugn = w * (r.a * gN.x + r.b * gN.y + gN.z);
        const float inv = 1.0f / rad;
        gx += ut * dtx + (dtx * ugn - w * gN.x) * inv;
        gy += ut * dty + (dty * ugn - w * gN.y) * inv;
        gz += ut * dtz + (dtz * ugn - w * gN.z) * inv;
        grr += ut * dtr + (ugn * dtr - w * (gN.x * o.n.x + gN.y * o.n.y + gN.z * o.n.z)) * inv;
      }
      const bool nz = gx != 0.0f || gy != 0.0f || gz != 0.0f || grr != 0.0f;
      if (__any_sync(0xffffffffu, nz)) {
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
          gx += __shfl_xor_sync(0xffffffffu, gx, off);
          gy += __shfl_xor_sync(0xffffffffu, gy, off);
          gz += __shfl_xor_sync(0xffffffffu, gz, off);
          grr += __shfl_xor_sync(0xffffffffu, grr, off);
        }
        if (lane == 0) {
          float *dst = grad + 4LL * pr.id;
          atomicAdd(dst + 0, v.R[0] * gx + v.U[0] * gy + v.F[0] * gz);
          atomicAdd(dst + 1, v.R[1] * gx + v.U[1] * gy + v.F[1] * gz);
          atomicAdd(dst + 2, v.R[2] * gx + v.U[2] * gy + v.F[2] * gz);
          atomicAdd(dst + 3, grr);
        }
      }
    }
  }
}

cudaError_t run_soft_pipeline(const Geometry &g, const Scene &sc, const Scratch &s, float *cov, float *depth,
                              float *normal, const float *g_cov, const float *g_depth, const float *g_normal,
                              float *grad, cudaStream_t st, StageEvents *evs) {
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_soft_fwd, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSoftSmem);
    cudaFuncSetAttribute(k_soft_bwd, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSoftSmem);
    attr = true;
  }
  cudaError_t e = run_binning(g, sc, s, st, evs, true);
  if (e != cudaSuccess) return e;
  const long long n_tiles = (long long)g.n_img * g.tiles_per_img;
  if (grad == nullptr) {
    k_soft_fwd<<<(unsigned)n_tiles, kSoftNT, kSoftSmem, st>>>(g, s.recs, s.rec_of, s.entries, s.cap_entries,
                                                             s.tile_count, s.tile_start, s.status, cov, depth,
                                                             normal);
  } else {
    cudaMemsetAsync(grad, 0, sizeof(float) * 4 * (size_t)g.n_atoms, st);
    k_soft_bwd<<<(unsigned)n_tiles, kSoftNT, kSoftSmem, st>>>(g, s.recs, s.rec_of, s.entries, s.cap_entries,
                                                             s.tile_count, s.tile_start, s.status, g_cov, g_depth,
                                                             g_normal, grad);
  }
  if (evs && evs->ev && evs->n > 5) cudaEventRecord(evs->ev[5], st);
  if (evs && evs->ev && evs->n > 6) cudaEventRecord(evs->ev[6], st);
  if (evs && evs->ev && evs->n > 7) cudaEventRecord(evs->ev[7], st);
  return cudaGetLastError();
}

}  // namespace vtx
