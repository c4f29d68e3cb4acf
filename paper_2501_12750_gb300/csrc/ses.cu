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
//   3. SES interior: edt2 >= 1 and edt2 h^2 >= p^2 (FP64; an integer threshold
//      here, as the product is monotone in edt2).  Marching cubes in two passes:
//      each CTA classifies a run of cells (one case byte per cell) and counts
//      their triangles, one CTA scans the counts, then each CTA writes its
//      cells' triangles in cell order, so the output order is deterministic.  The per-case
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
  int t_in;      // smallest edt2 with edt2 * h^2 >= p^2 in FP64 (the SES test, monotone in edt2)
  float xmax;    // largest |coordinate| of any grid point (bounds the FP32 rounding of the SAS filter)
};

__device__ __forceinline__ double grid_coord(float o, float h, long long i) {
  return __dadd_rn((double)o, __dmul_rn((double)h, (double)i));
}

// Set n bytes to 1: bytes up to a 4-byte boundary, then words, then bytes.
__device__ __forceinline__ void fill_ones(uint8_t *p, long long n) {
  while (n > 0 && ((uintptr_t)p & 3u)) {
    *p++ = 1;
    --n;
  }
  uint32_t *w = reinterpret_cast<uint32_t *>(p);
  for (; n >= 4; n -= 4) *w++ = 0x01010101u;
  p = reinterpret_cast<uint8_t *>(w);
  while (n-- > 0) *p++ = 1;
}

__device__ __forceinline__ bool sas_exact(const SesGrid &G, long long i, double dy2, double dz2, double cx, double R2) {
  const double dx = __dsub_rn(grid_coord(G.ox, G.h, i), cx);
  return __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), dy2), dz2) < R2;
}

// SAS interior: one warp per atom, lanes over the (j, k) rows of its box.
// Each point is first classified in FP32 with a bound M on the FP32 error of
// d^2 (coordinates, differences and squares, all at most a few ulps of
// numbers <= xmax + R + 2h, and of R^2 itself); only points within M of the
// sphere are decided by the exact FP64 test, so every decision equals the
// FP64 one.  Per row, only the points of the chord |dx|^2 <= R^2 - dy^2 -
// dz^2 + M are visited.
__global__ __launch_bounds__(256) void k_ses_sas(SesGrid G, const float4 *__restrict__ X, long long n,
                                                 uint8_t *__restrict__ sas) {
  const int lane = threadIdx.x & 31;
  const long long warp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const long long n_warps = ((long long)gridDim.x * blockDim.x) >> 5;
  for (long long a = warp; a < n; a += n_warps) {
    const float4 c = X[a];
    // FP32 throughout except on the rare points the filter cannot decide (the
    // FP64 pipes are a small fraction of the FP32 ones on this part)
    const float Rf = c.w + G.p, R2f = Rf * Rf;
    const float span = G.xmax + Rf + 2.0f * G.h;
    const float delta = 4e-7f * span;                      // |FP32 difference - exact| per axis
    const float ext = Rf + 2.0f * G.h;
    const float M = 8.0f * ext * delta + 4.0f * delta * delta + 1e-6f * ext * ext + 1e-6f;
    // candidate index ranges, two points wider than the sphere's extent on each side
    const float inv_h = 1.0f / G.h;
    long long lo[3], hi[3];
    const float cf[3] = {c.x, c.y, c.z};
    const float of[3] = {G.ox, G.oy, G.oz};
    const long long nn[3] = {G.nx, G.ny, G.nz};
    for (int d = 0; d < 3; ++d) {
      lo[d] = (long long)floorf((cf[d] - Rf - of[d]) * inv_h) - 2;
      hi[d] = (long long)ceilf((cf[d] + Rf - of[d]) * inv_h) + 2;
      lo[d] = lo[d] < 0 ? 0 : lo[d];
      hi[d] = hi[d] > nn[d] - 1 ? nn[d] - 1 : hi[d];
    }
    if (lo[0] > hi[0] || lo[1] > hi[1] || lo[2] > hi[2]) continue;
    const long long ny_box = hi[1] - lo[1] + 1;
    const long long rows = ny_box * (hi[2] - lo[2] + 1);
    for (long long r = lane; r < rows; r += 32) {
      const long long j = lo[1] + r % ny_box, k = lo[2] + r / ny_box;
      const float dyf = __fsub_rn(__fmaf_rn(G.h, (float)j, G.oy), c.y);
      const float dzf = __fsub_rn(__fmaf_rn(G.h, (float)k, G.oz), c.z);
      const float yz = __fmaf_rn(dyf, dyf, __fmul_rn(dzf, dzf));
      const float t = R2f - yz;
      if (t < -M) continue;  // the whole row is outside
      const float w = sqrtf(fmaxf(t + M, 0.0f)) + 2.0f * delta;
      long long i0 = (long long)floorf((c.x - w - G.ox) * inv_h) - 2, i1 = (long long)ceilf((c.x + w - G.ox) * inv_h) + 2;
      i0 = i0 < lo[0] ? lo[0] : i0;
      i1 = i1 > hi[0] ? hi[0] : i1;
      bool have64 = false;
      double dy2 = 0.0, dz2 = 0.0, R2 = 0.0;
      uint8_t *row = sas + (k * G.ny + j) * (long long)G.nx;
      // 1 = certainly inside, 0 = certainly outside, else the exact FP64 decision
      auto classify = [&](long long i, bool &certain) -> bool {
        const float dxf = __fsub_rn(__fmaf_rn(G.h, (float)i, G.ox), c.x);
        const float d2f = __fmaf_rn(dxf, dxf, yz);
        certain = d2f < R2f - M;
        if (certain) return true;
        if (d2f > R2f + M) return false;
        if (!have64) {
          const double dy = __dsub_rn(grid_coord(G.oy, G.h, j), (double)c.y);
          const double dz = __dsub_rn(grid_coord(G.oz, G.h, k), (double)c.z);
          dy2 = __dmul_rn(dy, dy);
          dz2 = __dmul_rn(dz, dz);
          const double R = __dadd_rn((double)c.w, (double)G.p);
          R2 = __dmul_rn(R, R);
          have64 = true;
        }
        return sas_exact(G, i, dy2, dz2, (double)c.x, R2);
      };
      // from each end of the chord, decide points one by one up to the first one
      // certainly inside; d^2 is convex along the row, so every point between the
      // two certain ones is inside with the same margin and is filled directly
      long long a_in = -1, b_in = -1;
      for (long long i = i0; i <= i1; ++i) {
        bool certain;
        if (classify(i, certain)) row[i] = 1;
        if (certain) {
          a_in = i;
          break;
        }
      }
      if (a_in >= 0) {
        for (long long i = i1; i > a_in; --i) {
          bool certain;
          if (classify(i, certain)) row[i] = 1;
          if (certain) {
            b_in = i;
            break;
          }
        }
        if (b_in > a_in + 1) fill_ones(row + a_in + 1, b_in - a_in - 1);
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



__device__ __forceinline__ int cell_case(const SesGrid &G, const uint16_t *__restrict__ edt, long long i, long long j,
                                         long long k) {
  int cs = 0;
#pragma unroll
  for (int c = 0; c < 8; ++c) {
    const long long q = ((k + c_corner[c][2]) * G.ny + (j + c_corner[c][1])) * (long long)G.nx + (i + c_corner[c][0]);
    if ((int)edt[q] >= G.t_in) cs |= 1 << c;
  }
  return cs;
}

// Triangles of the cells [c0, c0 + kSesCellsPerThread) of a thread; their cases
// are stored (one byte per cell) for the emit pass.
__device__ __forceinline__ int thread_cells_count(const SesGrid &G, const uint16_t *__restrict__ edt, long long c0,
                                                  long long n_cells, uint8_t *__restrict__ cases) {
  int n = 0;
  const long long cx = G.nx - 1, cy = G.ny - 1;
  for (int u = 0; u < kSesCellsPerThread; ++u) {
    const long long c = c0 + u;
    if (c >= n_cells) break;
    const long long i = c % cx, j = (c / cx) % cy, k = c / (cx * cy);
    const int cs = cell_case(G, edt, i, j, k);
    cases[c] = (uint8_t)cs;
    n += c_ses_case[cs].n_tris;
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
                                                           long long n_cells, uint8_t *__restrict__ cases,
                                                           unsigned *__restrict__ block_tris) {
  const long long c0 = (long long)blockIdx.x * kSesCellsPerBlock + (long long)threadIdx.x * kSesCellsPerThread;
  unsigned total;
  block_exclusive_sum((unsigned)thread_cells_count(G, edt, c0, n_cells, cases), &total);
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

// Vertex on edge e of cell (i, j, k): X_a + t (X_b - X_a), t = f_a / (f_a - f_b) clamped.
__device__ __forceinline__ float3 edge_vertex(const SesGrid &G, const uint16_t *__restrict__ edt, long long i,
                                              long long j, long long k, int e) {
  const int a = c_edge[e][0], b = c_edge[e][1];
  const long long ai = i + c_corner[a][0], aj = j + c_corner[a][1], ak = k + c_corner[a][2];
  const long long bi = i + c_corner[b][0], bj = j + c_corner[b][1], bk = k + c_corner[b][2];
  const float fa = sqrtf((float)edt[(ak * G.ny + aj) * (long long)G.nx + ai]) * G.h - G.p;
  const float fb = sqrtf((float)edt[(bk * G.ny + bj) * (long long)G.nx + bi]) * G.h - G.p;
  float s = fa == fb ? 0.5f : fa / (fa - fb);
  s = fminf(fmaxf(s, 0.0f), 1.0f);
  const float3 A = make_float3(G.ox + G.h * (float)ai, G.oy + G.h * (float)aj, G.oz + G.h * (float)ak);
  const float3 B = make_float3(G.ox + G.h * (float)bi, G.oy + G.h * (float)bj, G.oz + G.h * (float)bk);
  return make_float3(A.x + s * (B.x - A.x), A.y + s * (B.y - A.y), A.z + s * (B.z - A.z));
}

// One thread per output triangle of the CTA's run of cells: the cells'
// triangle offsets are scanned into shared memory, each thread finds its cell
// by binary search, its loop and fan position from the case table, and writes
// its triangle next to its neighbours' (coalesced).
__global__ __launch_bounds__(kSesThreads) void k_ses_emit(SesGrid G, const uint16_t *__restrict__ edt,
                                                          const uint8_t *__restrict__ cases, long long n_cells,
                                                          const unsigned long long *__restrict__ block_base,
                                                          float *__restrict__ tris, long long *__restrict__ labels,
                                                          unsigned long long max_tris) {
  __shared__ unsigned s_off[kSesCellsPerBlock + 1];
  __shared__ unsigned char s_case[kSesCellsPerBlock];
  const long long cb = (long long)blockIdx.x * kSesCellsPerBlock;
  unsigned n4[kSesCellsPerThread];
  unsigned mine = 0;
  for (int u = 0; u < kSesCellsPerThread; ++u) {
    const int lc = threadIdx.x * kSesCellsPerThread + u;
    const unsigned char cs = cb + lc < n_cells ? cases[cb + lc] : 0;
    s_case[lc] = cs;
    n4[u] = c_ses_case[cs].n_tris;
    mine += n4[u];
  }
  unsigned total;
  unsigned run = block_exclusive_sum(mine, &total);
  for (int u = 0; u < kSesCellsPerThread; ++u) {
    s_off[threadIdx.x * kSesCellsPerThread + u] = run;
    run += n4[u];
  }
  if (threadIdx.x == 0) s_off[kSesCellsPerBlock] = total;
  __syncthreads();
  const unsigned long long base_t = block_base[blockIdx.x];
  const long long cx = G.nx - 1, cy = G.ny - 1;
  for (unsigned q = threadIdx.x; q < total; q += kSesThreads) {
    int lo = 0, hi = kSesCellsPerBlock - 1;  // last cell with s_off <= q
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (s_off[mid] <= q) lo = mid; else hi = mid - 1;
    }
    const long long c = cb + lo;
    const SesCase &tc = c_ses_case[s_case[lo]];
    unsigned r = q - s_off[lo];
    int at = 0, l = 0;
    while (l < tc.n_loops) {
      const unsigned nt = tc.len[l] == 3 ? 1u : tc.len[l];
      if (r < nt) break;
      r -= nt;
      at += tc.len[l];
      ++l;
    }
    const long long i = c % cx, j = (c / cx) % cy, k = c / (cx * cy);
    const long long base = c * 16;
    const int L = tc.len[l];
    if (L == 3) {
      const int e0 = tc.edge[at], e1 = tc.edge[at + 1], e2 = tc.edge[at + 2];
      store_tri(tris, labels, base_t + q, max_tris, edge_vertex(G, edt, i, j, k, e0), edge_vertex(G, edt, i, j, k, e1),
                edge_vertex(G, edt, i, j, k, e2), base + e0, base + e1, base + e2);
    } else {
      float3 M = make_float3(0.0f, 0.0f, 0.0f);
      for (int v = 0; v < L; ++v) {
        const float3 p = edge_vertex(G, edt, i, j, k, tc.edge[at + v]);
        M.x += p.x;
        M.y += p.y;
        M.z += p.z;
      }
      const float inv = 1.0f / (float)L;
      M = make_float3(M.x * inv, M.y * inv, M.z * inv);
      const int q0 = (int)r, q1 = q0 + 1 == L ? 0 : q0 + 1;
      const int ea = tc.edge[at + q0], eb = tc.edge[at + q1];
      store_tri(tris, labels, base_t + q, max_tris, M, edge_vertex(G, edt, i, j, k, ea),
                edge_vertex(G, edt, i, j, k, eb), base + 12 + l, base + ea, base + eb);
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
            ses_window(L.probe, L.h), 1, 0.0f};
  {
    // SES interior <=> edt2 >= 1 (inside the SAS) and edt2 * h^2 >= p^2 in FP64: the product is monotone in
    // edt2, so the test is edt2 >= t_in for the smallest such integer
    const double hh = (double)L.h * (double)L.h, pp = (double)L.probe * (double)L.probe;
    long long t = (long long)std::floor(pp / hh);
    while (t > 0 && (double)(t - 1) * hh >= pp) --t;
    while ((double)t * hh < pp) ++t;
    G.t_in = (int)(t < 1 ? 1 : t);
    double xm = 0.0;
    for (int d = 0; d < 3; ++d) {
      const double a0 = std::fabs((double)L.origin[d]);
      const double a1 = std::fabs((double)L.origin[d] + (double)L.h * (double)(L.dims[d] - 1));
      xm = std::fmax(xm, std::fmax(a0, a1));
    }
    G.xmax = (float)(xm * 1.001 + 1.0);
  }
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
    k_ses_count<<<(unsigned)n_blocks, kSesThreads, 0, st>>>(G, L.edt2, n_cells, L.cases, L.block_tris);
    k_ses_scan<<<1, kSesThreads, 0, st>>>(L.block_tris, n_blocks, L.block_base, L.total);
    k_ses_emit<<<(unsigned)n_blocks, kSesThreads, 0, st>>>(G, L.edt2, L.cases, n_cells, L.block_base, L.tris,
                                                           L.labels, (unsigned long long)L.max_tris);
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
