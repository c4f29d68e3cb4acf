// static_vis.cu -- visibility buffer of one frame without any allocation.
//
// Some callers cannot allocate device memory at all: code running inside a
// host-side allocator or memory-pool callback, plug-ins of applications that
// own every allocation on the device, or real-time loops that forbid
// cudaMalloc's implicit synchronisation.  vtx_render_visibility_static()
// serves them: its scratch (the per-pixel 64-bit depth keys and the depth
// range) lives in one file-scope __device__ array of fixed size, so the call
// allocates nothing.  The caller passes device inputs and outputs.
//
// The kernels here are a compact variant of the frame pipeline: the same
// camera check and per-camera constants, conservative cull test, precise
// double-float setup and 64-bit atomicMin merge as the main path, but every
// surviving sphere is ray-cast directly over its candidate pixel box (no
// tile binning), which suits the small images this entry point is limited
// to; a box of more than 64 pixels is shared by the 32 lanes of a warp.
#include <mutex>

#include "../../include/vtx.h"
#include "vtx_internal.h"

namespace vtx {

// Scratch: [0, 4) image state words, [4, 4 + VTX_STATIC_MAX_PIXELS) keys.
constexpr long long kStaticHead = 4;
static __device__ __align__(256) unsigned long long g_static_scratch[kStaticHead + VTX_STATIC_MAX_PIXELS];

struct StaticHead {
  unsigned int zlo_bits, zhi_bits;
  float zlo, S;
  float invS;
  unsigned int valid;
  unsigned int pad[2];
};
static_assert(sizeof(StaticHead) <= kStaticHead * sizeof(unsigned long long), "head fits");

__global__ void k_static_clear(unsigned long long *scratch, long long n_px) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i == 0) {
    StaticHead *h = reinterpret_cast<StaticHead *>(scratch);
    h->zlo_bits = 0x7f800000u;
    h->zhi_bits = 0u;
    h->zlo = 0.0f;
    h->S = 0.0f;
    h->invS = 0.0f;
    h->valid = 0u;
  }
  for (long long p = i; p < n_px; p += (long long)gridDim.x * blockDim.x) scratch[kStaticHead + p] = kBgKey;
}

__device__ __forceinline__ bool static_cull(const ViewParams &v, float4 a, float &vx, float &vy, float &vz, float &Rm) {
  if (!(a.w >= 0.0f)) return false;
  float err;
  view_f32(v, a.x, a.y, a.z, vx, vy, vz, err);
  Rm = a.w + err;
  return cull_lean(v, vx, vy, vz, Rm);
}

__global__ void k_static_range(ViewParams v, const float4 *__restrict__ X, long long n, unsigned long long *scratch) {
  StaticHead *h = reinterpret_cast<StaticHead *>(scratch);
  float zlo = __int_as_float(0x7f800000), zhi = 0.0f;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    float vx, vy, vz, Rm;
    if (static_cull(v, X[i], vx, vy, vz, Rm)) {
      zlo = fminf(zlo, vz - Rm);
      zhi = fmaxf(zhi, vz + Rm);
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    zlo = fminf(zlo, __shfl_xor_sync(0xffffffffu, zlo, o));
    zhi = fmaxf(zhi, __shfl_xor_sync(0xffffffffu, zhi, o));
  }
  if ((threadIdx.x & 31) == 0 && zhi > 0.0f) {
    atomicMin(&h->zlo_bits, __float_as_uint(fmaxf(zlo, 0.0f)));
    atomicMax(&h->zhi_bits, __float_as_uint(zhi));
  }
}

__global__ void k_static_finalize(ViewParams v, unsigned long long *scratch) {
  StaticHead *h = reinterpret_cast<StaticHead *>(scratch);
  if (h->zhi_bits == 0u) {
    h->valid = 0u;
    return;
  }
  float lo = __uint_as_float(h->zlo_bits), hi = __uint_as_float(h->zhi_bits);
  lo = fmaxf(lo - 4e-6f * fabsf(lo) - 1e-4f, 0.5f * v.znear);
  hi = hi + 4e-6f * fabsf(hi) + 1e-4f;
  if (!(hi > lo)) hi = lo + 1.0f;
  h->zlo = lo;
  h->S = kKeySpanF / (hi - lo);
  h->invS = (hi - lo) / kKeySpanF;
  h->valid = 1u;
}

// Candidate boxes of more than kStaticBig pixels are ray-cast by the whole warp (lane l takes pixels
// l, l + 32, ...), so no thread tests more than ceil(W H / 32) pixels for one sphere, however close it is.
constexpr long long kStaticBig = 64;

__device__ __forceinline__ void static_hit(const ViewParams &v, int W, const Setup &su, float rad, uint32_t id,
                                           float S, int px, int py, unsigned long long *K) {
  const PixRay r = pix_ray(v, px, py);
  const float3 o = local_o(su.u0.hi, su.u0.lo, su.v0.hi, su.v0.lo, su.k, su.dz, r);
  float s;
  if (sphere_local(o, r, rad, s) && su.zr + s >= v.znear)
    atomicMin(K + (long long)py * W + px, pack_key(su.keyc, s, S, id));
}

__global__ void k_static_splat(ViewParams v, int W, int H, const float4 *__restrict__ X, long long n,
                               unsigned long long *scratch) {
  const StaticHead *h = reinterpret_cast<const StaticHead *>(scratch);
  if (!h->valid) return;
  const float zlo = h->zlo, S = h->S;
  unsigned long long *K = scratch + kStaticHead;
  const int lane = threadIdx.x & 31;
  const long long n_warps = ((long long)gridDim.x * blockDim.x) >> 5;
  // one atom per lane; the trip count is the same for all lanes of a warp
  for (long long w = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5; w * 32 < n; w += n_warps) {
    const long long i = w * 32 + lane;
    bool have = false;
    PixBox b{0, -1, 0, -1};
    Setup su;
    float rad = 0.0f;
    if (i < n) {
      const float4 a = X[i];
      float vx, vy, vz, Rm;
      if (static_cull(v, a, vx, vy, vz, Rm) && lean_box(v, W, H, vx, vy, vz, Rm, b)) {
        df dx, dy, dz;
        eye_offset(v, a, dx, dy, dz);
        su = precise_setup(v, dx, dy, dz, a.w, zlo, S);
        rad = a.w;
        have = true;
      }
    }
    const long long npx = have ? (long long)(b.x1 - b.x0 + 1) * (long long)(b.y1 - b.y0 + 1) : 0;
    const bool big = npx > kStaticBig;
    if (have && !big)
      for (int py = b.y0; py <= b.y1; ++py)
        for (int px = b.x0; px <= b.x1; ++px) static_hit(v, W, su, rad, (uint32_t)i, S, px, py, K);
    for (unsigned bigm = __ballot_sync(0xffffffffu, big); bigm != 0u; bigm &= bigm - 1u) {
      const int src = __ffs(bigm) - 1;
      Setup sb;
      sb.u0.hi = __shfl_sync(0xffffffffu, su.u0.hi, src);
      sb.u0.lo = __shfl_sync(0xffffffffu, su.u0.lo, src);
      sb.v0.hi = __shfl_sync(0xffffffffu, su.v0.hi, src);
      sb.v0.lo = __shfl_sync(0xffffffffu, su.v0.lo, src);
      sb.zr = __shfl_sync(0xffffffffu, su.zr, src);
      sb.dz = __shfl_sync(0xffffffffu, su.dz, src);
      sb.k = __shfl_sync(0xffffffffu, su.k, src);
      sb.keyc = __shfl_sync(0xffffffffu, su.keyc, src);
      const float rb = __shfl_sync(0xffffffffu, rad, src);
      const int x0 = __shfl_sync(0xffffffffu, b.x0, src), x1 = __shfl_sync(0xffffffffu, b.x1, src);
      const int y0 = __shfl_sync(0xffffffffu, b.y0, src), y1 = __shfl_sync(0xffffffffu, b.y1, src);
      const long long bw = x1 - x0 + 1, total = bw * (long long)(y1 - y0 + 1);
      const uint32_t id = (uint32_t)(w * 32 + src);
      for (long long q = lane; q < total; q += 32)
        static_hit(v, W, sb, rb, id, S, x0 + (int)(q % bw), y0 + (int)(q / bw), K);
    }
  }
}

__global__ void k_static_resolve(ViewParams v, int W, int H, const float4 *__restrict__ X,
                                 const unsigned long long *scratch, float *depth, uint32_t *idout) {
  const StaticHead *h = reinterpret_cast<const StaticHead *>(scratch);
  const int px = blockIdx.x * 32 + (threadIdx.x & 31);
  const int py = blockIdx.y * 8 + (threadIdx.x >> 5);
  if (px >= W || py >= H) return;
  const long long p = (long long)py * W + px;
  const unsigned long long key = scratch[kStaticHead + p];
  const uint32_t id = (uint32_t)key;
  if (id == kNoId) {
    depth[p] = __int_as_float(0x7f800000);
    idout[p] = kNoId;
    return;
  }
  const float4 a = X[id];
  df dx, dy, dz;
  eye_offset(v, a, dx, dy, dz);
  const Setup su = precise_setup(v, dx, dy, dz, a.w, h->zlo, h->S);
  const PixRay r = pix_ray(v, px, py);
  const float3 o = local_o(su.u0.hi, su.u0.lo, su.v0.hi, su.v0.lo, su.k, su.dz, r);
  const float ou = fmaf(o.x, r.a, fmaf(o.y, r.b, o.z));
  const float oo = fmaf(o.x, o.x, fmaf(o.y, o.y, o.z * o.z));
  const float disc = fmaxf(fmaf(ou, ou, -r.uu * (oo - a.w * a.w)), 0.0f);
  depth[p] = su.zr + (-ou - sqrtf(disc)) / r.uu;
  idout[p] = id;
}

}  // namespace vtx

using namespace vtx;

namespace {
std::mutex g_static_mu;
unsigned long long *g_static_ptr[64] = {};
}  // namespace

extern "C" vtx_status vtx_render_visibility_static(const float *xyzr, int64_t n_atoms, const vtx_camera *cam,
                                                   float *depth, uint32_t *id, void *cuda_stream) {
  if (!cam || !depth || !id || n_atoms < 0 || n_atoms > 2147483647LL || (n_atoms > 0 && !xyzr))
    return VTX_ERR_INVALID_ARG;
  if (((uintptr_t)xyzr & 15u) != 0) return VTX_ERR_INVALID_ARG;
  if (!cam_ok(cam)) return VTX_ERR_INVALID_ARG;  // the same camera check as vtx_set_camera
  const long long n_px = (long long)cam->width * cam->height;
  if (n_px > VTX_STATIC_MAX_PIXELS) return VTX_ERR_CAPACITY;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
    cudaGetLastError();
    return VTX_ERR_CUDA;
  }
  unsigned long long *scratch = nullptr;
  {
    // the array's device address, looked up once per device with that device current
    std::lock_guard<std::mutex> lock(g_static_mu);
    if (!g_static_ptr[dev]) {
      void *ptr = nullptr;
      if (cudaGetSymbolAddress(&ptr, g_static_scratch) != cudaSuccess || !ptr) {
        cudaGetLastError();
        return VTX_ERR_CUDA;
      }
      g_static_ptr[dev] = (unsigned long long *)ptr;
    }
    scratch = g_static_ptr[dev];
  }
  cudaStream_t st = (cudaStream_t)cuda_stream;
  const ViewParams v = make_view(*cam);  // the per-camera constants of the main path
  const int sms = sm_count();
  const float4 *X = (const float4 *)xyzr;
  const int ga = (int)(n_atoms / 256 + 1 < 8LL * sms ? n_atoms / 256 + 1 : 8LL * sms);
  k_static_clear<<<4 * sms, 256, 0, st>>>(scratch, n_px);
  k_static_range<<<ga, 256, 0, st>>>(v, X, n_atoms, scratch);
  k_static_finalize<<<1, 1, 0, st>>>(v, scratch);
  k_static_splat<<<ga, 256, 0, st>>>(v, cam->width, cam->height, X, n_atoms, scratch);
  dim3 grid((cam->width + 31) / 32, (cam->height + 7) / 8);
  k_static_resolve<<<grid, 256, 0, st>>>(v, cam->width, cam->height, X, scratch, depth, id);
  return cudaGetLastError() == cudaSuccess ? VTX_OK : VTX_ERR_CUDA;
}
