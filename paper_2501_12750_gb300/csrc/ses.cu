// ses.cu -- solvent excluded surface (SES) on a grid, extracted by marching
// cubes (Methods, "Cartoon and SES representations": a discrete approach in
// the manner of Lindow et al., surface by Lorensen-Cline marching cubes).
//
//   1. SAS interior: a grid point X = o + h (i, j, k) is inside when some atom
//      has ((X-c)_x^2 + (X-c)_y^2) + (X-c)_z^2 < (r + p)^2, evaluated in FP64
//      with every operation explicitly rounded (no contraction), so the
//      decision is a pure function of the inputs.  One warp per atom, one
//      lane per grid row of the atom's box.
//   2. Squared distance (grid units) to the nearest point outside the SAS
//      interior, exact inside a (2K+1)^3 window (K = ceil(p/h) + 1) and
//      K^2 + 1 beyond: three separable min-plus passes (x, y, z), integers
//      only.  Marching cubes only ever needs values <= K^2.
//   3. SES interior: edt2 h^2 >= p^2 (FP64).  Marching cubes in two passes:
//      each CTA counts the triangles of a run of cells, one CTA scans the
//      counts, then each CTA re-derives its cells and writes their triangles
//      in cell order, so the output order is deterministic.  The per-case
//      loops come from a table built once on the host: faces with four
//      crossings cut their inside corners apart, segments are directed by the
//      face's outward normal so loops turn counter-clockwise about the
//      outward (inside to outside) normal, and loops longer than three edges
//      become a star of triangles around their mean vertex.
#include <cmath>
#include <mutex>

#include "vtx_internal.h"

namespace vtx {

constexpr int kSesThreads = 256;
constexpr int kSesCellsPerThread = 4;
constexpr int kSesCellsPerBlock = kSesThreads * kSesCellsPerThread;
constexpr uint16_t kSesInf = 0xffffu;

// Per case: number of loops, their lengths, and their edges back to back.
struct SesCase {
  unsigned char n_loops;
  unsigned char n_tris;
  unsigned char len[4];
  unsigned char edge[12];
};
__constant__ SesCase c_ses_case[256];

// Corners (x, y, z offsets) and edges (corner pairs) of a cell.
__constant__ int c_corner[8][3] = {{0, 0, 0}, {1, 0, 0}, {1, 1, 0}, {0, 1, 0}, {0, 0, 1}, {1, 0, 1}, {1, 1, 1}, {0, 1, 1}};
__constant__ int c_edge[12][2] = {{0, 1}, {1, 2}, {2, 3}, {3, 0}, {4, 5}, {5, 6},
                                  {6, 7}, {7, 4}, {0, 4}, {1, 5}, {2, 6}, {3, 7}};

// ------------------------------------------------------------ case table --

namespace {

const int kCorner[8][3] = {{0, 0, 0}, {1, 0, 0}, {1, 1, 0}, {0, 1, 0}, {0, 0, 1}, {1, 0, 1}, {1, 1, 1}, {0, 1, 1}};
const int kEdge[12][2] = {{0, 1}, {1, 2}, {2, 3}, {3, 0}, {4, 5}, {5, 6}, {6, 7}, {7, 4}, {0, 4}, {1, 5}, {2, 6}, {3, 7}};
// Faces: corner cycle and outward normal.
const int kFace[6][4] = {{0, 3, 2, 1}, {4, 5, 6, 7}, {0, 1, 5, 4}, {2, 3, 7, 6}, {0, 4, 7, 3}, {1, 2, 6, 5}};
const int kFaceN[6][3] = {{0, 0, -1}, {0, 0, 1}, {0, -1, 0}, {0, 1, 0}, {-1, 0, 0}, {1, 0, 0}};

int edge_between(int a, int b) {
  for (int e = 0; e < 12; ++e)
    if ((kEdge[e][0] == a && kEdge[e][1] == b) || (kEdge[e][1] == a && kEdge[e][0] == b)) return e;
  return -1;
}

// Twice the midpoint of edge e (integral).
void mid2(int e, long m[3]) {
  for (int k = 0; k < 3; ++k) m[k] = kCorner[kEdge[e][0]][k] + kCorner[kEdge[e][1]][k];
}

// Link crossing edges ea and eb on face f, the segment cutting off the inside
// corners cut[0..nc): direction d = m x n, m from the cut corners' mean to
// the segment's midpoint (all scaled to integers).
void link(int f, int ea, int eb, const int *cut, int nc, int next[12]) {
  long pa[3], pb[3], m[3];
  mid2(ea, pa);
  mid2(eb, pb);
  for (int k = 0; k < 3; ++k) {
    long c = 0;
    for (int q = 0; q < nc; ++q) c += 2 * kCorner[cut[q]][k];
    m[k] = (pa[k] + pb[k]) * nc - 2 * c;
  }
  const int *n = kFaceN[f];
  const long d[3] = {m[1] * n[2] - m[2] * n[1], m[2] * n[0] - m[0] * n[2], m[0] * n[1] - m[1] * n[0]};
  const long along = (pb[0] - pa[0]) * d[0] + (pb[1] - pa[1]) * d[1] + (pb[2] - pa[2]) * d[2];
  if (along > 0)
    next[ea] = eb;
  else
    next[eb] = ea;
}

SesCase build_case(int cs) {
  SesCase out{};
  if (cs == 0 || cs == 255) return out;
  int next[12];
  for (int e = 0; e < 12; ++e) next[e] = -1;
  for (int f = 0; f < 6; ++f) {
    const int *q = kFace[f];
    int crossing[4], n_cross = 0, in_c[4], n_in = 0;
    for (int s = 0; s < 4; ++s) {
      const bool a_in = (cs >> q[s]) & 1, b_in = (cs >> q[(s + 1) % 4]) & 1;
      if (a_in != b_in) crossing[n_cross++] = edge_between(q[s], q[(s + 1) % 4]);
      if (a_in) in_c[n_in++] = q[s];
    }
    if (n_cross == 2) {
      link(f, crossing[0], crossing[1], in_c, n_in, next);
    } else if (n_cross == 4) {
      for (int s = 0; s < 4; ++s)
        if ((cs >> q[s]) & 1) {
          const int c = q[s];
          link(f, edge_between(q[(s + 3) % 4], c), edge_between(c, q[(s + 1) % 4]), &c, 1, next);
        }
    }
  }
  bool seen[12] = {};
  int at = 0;
  for (int s = 0; s < 12; ++s) {
    if (next[s] < 0 || seen[s]) continue;
    int L = 0;
    for (int e = s; !seen[e]; e = next[e]) {
      seen[e] = true;
      out.edge[at + L++] = (unsigned char)e;
    }
    out.len[out.n_loops++] = (unsigned char)L;
    out.n_tris += (unsigned char)(L == 3 ? 1 : L);
    at += L;
  }
  return out;
}

std::once_flag g_table_once[64];
bool g_table_ok[64];

}  // namespace

// Upload the case table to this device's constant memory (once per device).
static bool ses_table_ready(int device) {
  if (device < 0 || device >= 64) return false;
  std::call_once(g_table_once[device], [device] {
    SesCase t[256];
    for (int cs = 0; cs < 256; ++cs) t[cs] = build_case(cs);
    g_table_ok[device] = cudaMemcpyToSymbol(c_ses_case, t, sizeof(t)) == cudaSuccess;
  });
  return g_table_ok[device];
}

// --------------------------------------------------------------- kernels --

struct SesGrid {
  float ox, oy, oz, h, p;
  int nx, ny, nz;
  int K;
};

__device__ __forceinline__ double grid_coord(float o, float h, long long i) {
  return __dadd_rn((double)o, __dmul_rn((double)h, (double)i));
}

// SAS interior: one warp per atom, lanes over the (j, k) rows of its box.
__global__ __launch_bounds__(256) void k_ses_sas(SesGrid G, const float4 *__restrict__ X, long long n,
                                                 uint8_t *__restrict__ sas) {
  const int lane = threadIdx.x & 31;
  const long long warp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const long long n_warps = ((long long)gridDim.x * blockDim.x) >> 5;
  for (long long a = warp; a < n; a += n_warps) {
    const float4 c = X[a];
    const double R = __dadd_rn((double)c.w, (double)G.p);
    const double R2 = __dmul_rn(R, R);
    // candidate index ranges, one point wider than the sphere's extent on each side
    const double hh = (double)G.h;
    long long lo[3], hi[3];
    const double cc[3] = {(double)c.x, (double)c.y, (double)c.z};
    const double oo[3] = {(double)G.ox, (double)G.oy, (double)G.oz};
    const long long nn[3] = {G.nx, G.ny, G.nz};
    for (int d = 0; d < 3; ++d) {
      lo[d] = (long long)floor((cc[d] - R - oo[d]) / hh) - 1;
      hi[d] = (long long)ceil((cc[d] + R - oo[d]) / hh) + 1;
      lo[d] = lo[d] < 0 ? 0 : lo[d];
      hi[d] = hi[d] > nn[d] - 1 ? nn[d] - 1 : hi[d];
    }
    if (lo[0] > hi[0] || lo[1] > hi[1] || lo[2] > hi[2]) continue;
    const long long ny_box = hi[1] - lo[1] + 1;
    const long long rows = ny_box * (hi[2] - lo[2] + 1);
    for (long long r = lane; r < rows; r += 32) {
      const long long j = lo[1] + r % ny_box, k = lo[2] + r / ny_box;
      const double dy = __dsub_rn(grid_coord(G.oy, G.h, j), cc[1]);
      const double dz = __dsub_rn(grid_coord(G.oz, G.h, k), cc[2]);
      const double dy2 = __dmul_rn(dy, dy), dz2 = __dmul_rn(dz, dz);
      uint8_t *row = sas + (k * G.ny + j) * (long long)G.nx;
      for (long long i = lo[0]; i <= hi[0]; ++i) {
        const double dx = __dsub_rn(grid_coord(G.ox, G.h, i), cc[0]);
        const double d2 = __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), dy2), dz2);
        if (d2 < R2) row[i] = 1;
      }
    }
  }
}

// Pass x: distance^2 along x to the nearest point outside the SAS interior, within K.
__global__ __launch_bounds__(256) void k_ses_edt_x(SesGrid G, const uint8_t *__restrict__ sas,
                                                   uint16_t *__restrict__ g1, long long n_pts) {
  for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < n_pts;
       q += (long long)gridDim.x * blockDim.x) {
    const long long i = q % G.nx;
    uint16_t best = kSesInf;
    if (!sas[q]) {
      best = 0;
    } else {
      for (int d = 1; d <= G.K; ++d) {
        const bool l = i - d >= 0 && !sas[q - d], r = i + d < G.nx && !sas[q + d];
        if (l || r) {
          best = (uint16_t)(d * d);
          break;
        }
      }
    }
    g1[q] = best;
  }
}

// Passes y and z: min over |d| <= K of d^2 + src[q + d * stride] (kSesInf = none).
// The last pass maps values above K^2 to the sentinel K^2 + 1.
__global__ __launch_bounds__(256) void k_ses_edt_yz(SesGrid G, const uint16_t *__restrict__ src,
                                                    uint16_t *__restrict__ dst, long long n_pts, long long stride,
                                                    long long extent, int last) {
  const int K2 = G.K * G.K;
  for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < n_pts;
       q += (long long)gridDim.x * blockDim.x) {
    const long long c = (q / stride) % extent;
    int best = src[q] == kSesInf ? 0x7fffffff : (int)src[q];
    for (int d = 1; d <= G.K; ++d) {
      const int dd = d * d;
      if (dd >= best) break;
      if (c - d >= 0) {
        const uint16_t v = src[q - d * stride];
        if (v != kSesInf && dd + (int)v < best) best = dd + (int)v;
      }
      if (c + d < extent) {
        const uint16_t v = src[q + d * stride];
        if (v != kSesInf && dd + (int)v < best) best = dd + (int)v;
      }
    }
    if (last)
      dst[q] = (uint16_t)(best > K2 ? K2 + 1 : best);
    else
      dst[q] = (uint16_t)(best > 0xfffe ? kSesInf : best);
  }
}

__device__ __forceinline__ bool ses_inside(uint16_t e, float h, float p) {
  return __dmul_rn((double)e, __dmul_rn((double)h, (double)h)) >= __dmul_rn((double)p, (double)p);
}

__device__ __forceinline__ int cell_case(const SesGrid &G, const uint16_t *__restrict__ edt, long long i, long long j,
                                         long long k) {
  int cs = 0;
#pragma unroll
  for (int c = 0; c < 8; ++c) {
    const long long q = ((k + c_corner[c][2]) * G.ny + (j + c_corner[c][1])) * (long long)G.nx + (i + c_corner[c][0]);
    if (ses_inside(edt[q], G.h, G.p)) cs |= 1 << c;
  }
  return cs;
}

// Triangles of the cells [c0, c0 + kSesCellsPerThread) of thread t: their count.
__device__ __forceinline__ int thread_cells_count(const SesGrid &G, const uint16_t *__restrict__ edt, long long c0,
                                                  long long n_cells) {
  int n = 0;
  const long long cx = G.nx - 1, cy = G.ny - 1;
  for (int u = 0; u < kSesCellsPerThread; ++u) {
    const long long c = c0 + u;
    if (c >= n_cells) break;
    const long long i = c % cx, j = (c / cx) % cy, k = c / (cx * cy);
    n += c_ses_case[cell_case(G, edt, i, j, k)].n_tris;
  }
  return n;
}

__device__ __forceinline__ unsigned block_exclusive_sum(unsigned v, unsigned *total) {
  __shared__ unsigned s_warp[kSesThreads / 32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  unsigned x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const unsigned y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) s_warp[w] = x;
  __syncthreads();
  if (w == 0) {
    unsigned s = lane < kSesThreads / 32 ? s_warp[lane] : 0u;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned y = __shfl_up_sync(0xffffffffu, s, o);
      if (lane >= o) s += y;
    }
    if (lane < kSesThreads / 32) s_warp[lane] = s;
  }
  __syncthreads();
  const unsigned before = (w > 0 ? s_warp[w - 1] : 0u) + x - v;
  if (total) *total = s_warp[kSesThreads / 32 - 1];
  __syncthreads();
  return before;
}

__global__ __launch_bounds__(kSesThreads) void k_ses_count(SesGrid G, const uint16_t *__restrict__ edt,
                                                           long long n_cells, unsigned *__restrict__ block_tris) {
  const long long c0 = (long long)blockIdx.x * kSesCellsPerBlock + (long long)threadIdx.x * kSesCellsPerThread;
  unsigned total;
  block_exclusive_sum((unsigned)thread_cells_count(G, edt, c0, n_cells), &total);
  if (threadIdx.x == 0) block_tris[blockIdx.x] = total;
}

// Exclusive scan of the per-block counts in one CTA (64-bit totals).
__global__ __launch_bounds__(kSesThreads) void k_ses_scan(const unsigned *__restrict__ block_tris, long long n_blocks,
                                                          unsigned long long *__restrict__ block_base,
                                                          unsigned long long *__restrict__ total) {
  __shared__ unsigned long long s_carry;
  if (threadIdx.x == 0) s_carry = 0ull;
  __syncthreads();
  for (long long b0 = 0; b0 < n_blocks; b0 += kSesThreads) {
    const long long b = b0 + threadIdx.x;
    const unsigned v = b < n_blocks ? block_tris[b] : 0u;
    unsigned tot;
    const unsigned ex = block_exclusive_sum(v, &tot);
    if (b < n_blocks) block_base[b] = s_carry + ex;
    __syncthreads();
    if (threadIdx.x == 0) s_carry += tot;
    __syncthreads();
  }
  if (threadIdx.x == 0) *total = s_carry;
}

__device__ __forceinline__ void store_tri(float *__restrict__ tris, long long *__restrict__ labels,
                                          unsigned long long t, unsigned long long max_tris, const float3 &a,
                                          const float3 &b, const float3 &c, long long la, long long lb, long long lc) {
  if (t >= max_tris) return;
  float *o = tris + t * 9;
  o[0] = a.x, o[1] = a.y, o[2] = a.z;
  o[3] = b.x, o[4] = b.y, o[5] = b.z;
  o[6] = c.x, o[7] = c.y, o[8] = c.z;
  if (labels) {
    labels[t * 3] = la;
    labels[t * 3 + 1] = lb;
    labels[t * 3 + 2] = lc;
  }
}

__global__ __launch_bounds__(kSesThreads) void k_ses_emit(SesGrid G, const uint16_t *__restrict__ edt,
                                                          long long n_cells,
                                                          const unsigned long long *__restrict__ block_base,
                                                          float *__restrict__ tris, long long *__restrict__ labels,
                                                          unsigned long long max_tris) {
  const long long c0 = (long long)blockIdx.x * kSesCellsPerBlock + (long long)threadIdx.x * kSesCellsPerThread;
  const unsigned before = block_exclusive_sum((unsigned)thread_cells_count(G, edt, c0, n_cells), nullptr);
  unsigned long long t = block_base[blockIdx.x] + before;
  const long long cx = G.nx - 1, cy = G.ny - 1;
  for (int u = 0; u < kSesCellsPerThread; ++u) {
    const long long c = c0 + u;
    if (c >= n_cells) break;
    const long long i = c % cx, j = (c / cx) % cy, k = c / (cx * cy);
    const int cs = cell_case(G, edt, i, j, k);
    const SesCase &tc = c_ses_case[cs];
    if (tc.n_tris == 0) continue;
    float f[8];
    float3 P[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const long long a = i + c_corner[q][0], b = j + c_corner[q][1], d = k + c_corner[q][2];
      const uint16_t e = edt[(d * G.ny + b) * (long long)G.nx + a];
      f[q] = sqrtf((float)e) * G.h - G.p;
      P[q] = make_float3(G.ox + G.h * (float)a, G.oy + G.h * (float)b, G.oz + G.h * (float)d);
    }
    int at = 0;
    for (int l = 0; l < tc.n_loops; ++l) {
      const int L = tc.len[l];
      float3 V[12];
      float3 M = make_float3(0.0f, 0.0f, 0.0f);
      for (int q = 0; q < L; ++q) {
        const int e = tc.edge[at + q], a = c_edge[e][0], b = c_edge[e][1];
        float s = f[a] == f[b] ? 0.5f : f[a] / (f[a] - f[b]);
        s = fminf(fmaxf(s, 0.0f), 1.0f);
        V[q] = make_float3(P[a].x + s * (P[b].x - P[a].x), P[a].y + s * (P[b].y - P[a].y), P[a].z + s * (P[b].z - P[a].z));
        M.x += V[q].x;
        M.y += V[q].y;
        M.z += V[q].z;
      }
      const long long base = c * 16;
      if (L == 3) {
        store_tri(tris, labels, t++, max_tris, V[0], V[1], V[2], base + tc.edge[at], base + tc.edge[at + 1],
                  base + tc.edge[at + 2]);
      } else {
        const float inv = 1.0f / (float)L;
        M = make_float3(M.x * inv, M.y * inv, M.z * inv);
        for (int q = 0; q < L; ++q) {
          const int q1 = q + 1 == L ? 0 : q + 1;
          store_tri(tris, labels, t++, max_tris, M, V[q], V[q1], base + 12 + l, base + tc.edge[at + q],
                    base + tc.edge[at + q1]);
        }
      }
      at += L;
    }
  }
}

// Bounding box of the SAS spheres: min and max of c -/+ (r + p), as float bits of
// non-negative-shifted values would be awkward, so each CTA reduces and writes one
// partial; the host finishes the (small) reduction.
__global__ __launch_bounds__(256) void k_ses_bbox(const float4 *__restrict__ X, long long n, float p,
                                                  float *__restrict__ partial) {
  float lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
  for (long long a = (long long)blockIdx.x * blockDim.x + threadIdx.x; a < n; a += (long long)gridDim.x * blockDim.x) {
    const float4 c = X[a];
    const float R = c.w + p;
    lo[0] = fminf(lo[0], c.x - R), hi[0] = fmaxf(hi[0], c.x + R);
    lo[1] = fminf(lo[1], c.y - R), hi[1] = fmaxf(hi[1], c.y + R);
    lo[2] = fminf(lo[2], c.z - R), hi[2] = fmaxf(hi[2], c.z + R);
  }
  __shared__ float s[6][8];
  for (int d = 0; d < 3; ++d) {
    for (int o = 16; o > 0; o >>= 1) {
      lo[d] = fminf(lo[d], __shfl_xor_sync(0xffffffffu, lo[d], o));
      hi[d] = fmaxf(hi[d], __shfl_xor_sync(0xffffffffu, hi[d], o));
    }
  }
  const int w = threadIdx.x >> 5;
  if ((threadIdx.x & 31) == 0)
    for (int d = 0; d < 3; ++d) {
      s[d][w] = lo[d];
      s[3 + d][w] = hi[d];
    }
  __syncthreads();
  if (threadIdx.x < 6) {
    float v = s[threadIdx.x][0];
    for (int q = 1; q < 8; ++q) v = threadIdx.x < 3 ? fminf(v, s[threadIdx.x][q]) : fmaxf(v, s[threadIdx.x][q]);
    partial[blockIdx.x * 6 + threadIdx.x] = v;
  }
}

// ------------------------------------------------------------- launchers --

int ses_window(float probe, float h) { return (int)std::ceil((double)probe / (double)h) + 1; }

cudaError_t run_ses_bbox(const float4 *X, long long n, float probe, float *partial, int n_blocks, cudaStream_t st) {
  k_ses_bbox<<<n_blocks, 256, 0, st>>>(X, n, probe, partial);
  return cudaGetLastError();
}

cudaError_t run_ses_grid(const SesLaunch &L, cudaStream_t st) {
  int dev = 0;
  cudaGetDevice(&dev);
  if (!ses_table_ready(dev)) return cudaErrorInvalidValue;
  SesGrid G{L.origin[0], L.origin[1], L.origin[2], L.h, L.probe, L.dims[0], L.dims[1], L.dims[2],
            ses_window(L.probe, L.h)};
  const long long n_pts = (long long)G.nx * G.ny * G.nz;
  const int sms = sm_count();
  cudaError_t e = cudaMemsetAsync(L.sas, 0, (size_t)n_pts, st);
  if (e != cudaSuccess) return e;
  if (L.n_atoms > 0) {
    const long long warps = L.n_atoms < 64LL * sms * 8 ? L.n_atoms : 64LL * sms * 8;
    k_ses_sas<<<(int)((warps * 32 + 255) / 256), 256, 0, st>>>(G, L.X, L.n_atoms, L.sas);
  }
  const long long pb = (n_pts + 255) / 256;
  const int grid = (int)(pb < 16LL * sms ? pb : 16LL * sms);
  k_ses_edt_x<<<grid, 256, 0, st>>>(G, L.sas, L.g_a, n_pts);
  k_ses_edt_yz<<<grid, 256, 0, st>>>(G, L.g_a, L.g_b, n_pts, (long long)G.nx, (long long)G.ny, 0);
  k_ses_edt_yz<<<grid, 256, 0, st>>>(G, L.g_b, L.edt2, n_pts, (long long)G.nx * G.ny, (long long)G.nz, 1);
  const long long n_cells = (long long)(G.nx - 1) * (G.ny - 1) * (G.nz - 1);
  const long long n_blocks = (n_cells + kSesCellsPerBlock - 1) / kSesCellsPerBlock;
  if (n_blocks > 0) {
    k_ses_count<<<(unsigned)n_blocks, kSesThreads, 0, st>>>(G, L.edt2, n_cells, L.block_tris);
    k_ses_scan<<<1, kSesThreads, 0, st>>>(L.block_tris, n_blocks, L.block_base, L.total);
    k_ses_emit<<<(unsigned)n_blocks, kSesThreads, 0, st>>>(G, L.edt2, n_cells, L.block_base, L.tris, L.labels,
                                                           (unsigned long long)L.max_tris);
  } else {
    cudaMemsetAsync(L.total, 0, sizeof(unsigned long long), st);
  }
  return cudaGetLastError();
}

long long ses_blocks(const int32_t dims[3]) {
  const long long n_cells = (long long)(dims[0] - 1) * (dims[1] - 1) * (dims[2] - 1);
  return (n_cells + kSesCellsPerBlock - 1) / kSesCellsPerBlock;
}

}  // namespace vtx
