/*
 * ses_oracle.c -- CPU FP64 oracle of the solvent excluded surface (SES) by a
 * discrete grid and marching cubes (Methods, "Cartoon and SES
 * representations": the SES is computed on a grid, in the manner of Lindow
 * et al., and its surface extracted by marching cubes, Lorensen and Cline).
 *
 * TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).  Plain loops over every
 * grid point and every atom; no code is shared with the renderer.
 *
 * Definitions (the paper names the method only; these are the readings):
 *
 *   Grid point (i, j, k) sits at X = (o + h i, o + h j, o + h k), evaluated in
 *   FP64 as (double)o_x + (double)h * i.
 *
 *   SAS interior: X is inside when, for some atom c with radius r,
 *   ((X-c)_x^2 + (X-c)_y^2) + (X-c)_z^2  <  (r + p)^2, every operation a
 *   correctly rounded FP64 operation in exactly this order (R = (double)r +
 *   (double)p, R^2 = R * R).
 *
 *   Distance to the probe-accessible region: edt2(X) = the squared distance,
 *   in grid units, from X to the nearest grid point outside the SAS interior,
 *   if that is <= K^2 with K = ceil(p / h) + 1; otherwise the sentinel
 *   K^2 + 1 ("farther").  0 for points outside the SAS interior.
 *
 *   SES interior: edt2 > 0 and edt2 * h^2 >= p^2 (FP64: (double)edt2 *
 *   ((double)h * (double)h) >= (double)p * (double)p): inside the SAS and no
 *   probe centre within p (with p = 0 the SES is the SAS, the union of the
 *   spheres).
 *   Field for interpolation: f = sqrt(edt2) h - p (>= 0 inside).
 *
 *   Marching cubes: cell (i, j, k) spans grid points (i..i+1, j..j+1, k..k+1),
 *   corners numbered 0 (0,0,0), 1 (1,0,0), 2 (1,1,0), 3 (0,1,0), 4 (0,0,1),
 *   5 (1,0,1), 6 (1,1,1), 7 (0,1,1); edges 0 (0-1), 1 (1-2), 2 (2-3), 3 (3-0),
 *   4 (4-5), 5 (5-6), 6 (6-7), 7 (7-4), 8 (0-4), 9 (1-5), 10 (2-6), 11 (3-7).
 *   Case bit c is set when corner c is inside the SES.  On every face the
 *   crossing edges are joined by segments; a face with four crossings (two
 *   diagonal inside corners) cuts each inside corner off on its own.  The
 *   segments are directed along m x n_f (m from the face's cut-off inside
 *   corners to the segment, n_f the face's outward normal), so every loop
 *   runs counter-clockwise about the normal pointing from inside to outside.
 *   Each loop starts at its smallest edge number; loops are emitted in order
 *   of their first edge; a loop of three edges is one triangle (l0, l1, l2),
 *   a longer loop of L edges is L triangles (m, l_q, l_q+1) around m, the
 *   mean of its L vertices (a fan from one loop vertex could lay a triangle
 *   flat in a cube face, doubled by the neighbouring cell); cells in order i
 *   fastest, then j, then k.  The vertex on edge (a, b) is X_a + t (X_b -
 *   X_a), t = f_a / (f_a - f_b), clamped to [0, 1].  Vertex labels: cell * 16
 *   + edge for edge vertices, cell * 16 + 12 + loop for loop means.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#include <omp.h>

static const int SES_CORNER[8][3] = {{0, 0, 0}, {1, 0, 0}, {1, 1, 0}, {0, 1, 0},
                                     {0, 0, 1}, {1, 0, 1}, {1, 1, 1}, {0, 1, 1}};
static const int SES_EDGE[12][2] = {{0, 1}, {1, 2}, {2, 3}, {3, 0}, {4, 5}, {5, 6},
                                    {6, 7}, {7, 4}, {0, 4}, {1, 5}, {2, 6}, {3, 7}};
/* faces as corner cycles (any consistent cycle works: only adjacency is used) */
static const int SES_FACE[6][4] = {{0, 1, 2, 3}, {4, 5, 6, 7}, {0, 1, 5, 4},
                                   {3, 2, 6, 7}, {0, 3, 7, 4}, {1, 2, 6, 5}};

static int edge_of(int a, int b) {
  for (int e = 0; e < 12; ++e)
    if ((SES_EDGE[e][0] == a && SES_EDGE[e][1] == b) || (SES_EDGE[e][0] == b && SES_EDGE[e][1] == a)) return e;
  return -1;
}

/* offset (nullable): grid index of this array's first point in a larger grid with the same origin. */
void orc_ses_sas(const float *xyzr, int64_t n_atoms, float probe, const float *origin, float h, const int32_t *dims,
                 const int32_t *offset, uint8_t *inside) {
  const int64_t nx = dims[0], ny = dims[1], nz = dims[2];
  const int64_t o0 = offset ? offset[0] : 0, o1 = offset ? offset[1] : 0, o2 = offset ? offset[2] : 0;
#pragma omp parallel for schedule(dynamic, 1)
  for (int64_t k = 0; k < nz; ++k)
    for (int64_t j = 0; j < ny; ++j)
      for (int64_t i = 0; i < nx; ++i) {
        const double X = (double)origin[0] + (double)h * (double)(i + o0);
        const double Y = (double)origin[1] + (double)h * (double)(j + o1);
        const double Z = (double)origin[2] + (double)h * (double)(k + o2);
        uint8_t in = 0;
        for (int64_t a = 0; a < n_atoms && !in; ++a) {
          const float *c = xyzr + 4 * a;
          const double R = (double)c[3] + (double)probe;
          const double dx = X - (double)c[0], dy = Y - (double)c[1], dz = Z - (double)c[2];
          const double d2 = (dx * dx + dy * dy) + dz * dz;
          if (d2 < R * R) in = 1;
        }
        inside[(k * ny + j) * nx + i] = in;
      }
}

int32_t orc_ses_k(float probe, float h) { return (int32_t)ceil((double)probe / (double)h) + 1; }

void orc_ses_edt(const uint8_t *inside, const int32_t *dims, int32_t K, uint16_t *edt2) {
  const int64_t nx = dims[0], ny = dims[1], nz = dims[2];
  const int32_t far = K * K + 1;
#pragma omp parallel for schedule(dynamic, 1)
  for (int64_t k = 0; k < nz; ++k)
    for (int64_t j = 0; j < ny; ++j)
      for (int64_t i = 0; i < nx; ++i) {
        int32_t best = far;
        if (!inside[(k * ny + j) * nx + i]) {
          best = 0;
        } else {
          for (int64_t c = k - K; c <= k + K; ++c)
            for (int64_t b = j - K; b <= j + K; ++b)
              for (int64_t a = i - K; a <= i + K; ++a) {
                if (a < 0 || b < 0 || c < 0 || a >= nx || b >= ny || c >= nz) continue;
                if (inside[(c * ny + b) * nx + a]) continue;
                const int32_t d = (int32_t)((a - i) * (a - i) + (b - j) * (b - j) + (c - k) * (c - k));
                if (d < best) best = d;
              }
          if (best > K * K) best = far;
        }
        edt2[(k * ny + j) * nx + i] = (uint16_t)best;
      }
}

static int ses_in(uint16_t e, float h, float p) {
  return e > 0 && (double)e * ((double)h * (double)h) >= (double)p * (double)p;
}

/* Outward normals of the faces above (corner coordinates are 0/1). */
static const int SES_FACE_N[6][3] = {{0, 0, -1}, {0, 0, 1}, {0, -1, 0}, {0, 1, 0}, {-1, 0, 0}, {1, 0, 0}};

/*
 * Directed segment on face f between crossing edges ea and eb, cutting off
 * the face corners listed in side[0..ns) (the inside ones).  The segment is
 * directed along d = m x n_f, m pointing from those corners to the segment,
 * so that every loop runs counter-clockwise about the outward (inside to
 * outside) normal.  Coordinates are doubled to stay integral.
 */
static void add_segment(int f, int ea, int eb, const int *side, int ns, int *succ) {
  long ma[3], mb[3], cen[3] = {0, 0, 0}, m[3], dvec[3];
  for (int k = 0; k < 3; ++k) {
    ma[k] = SES_CORNER[SES_EDGE[ea][0]][k] + SES_CORNER[SES_EDGE[ea][1]][k];
    mb[k] = SES_CORNER[SES_EDGE[eb][0]][k] + SES_CORNER[SES_EDGE[eb][1]][k];
  }
  for (int q = 0; q < ns; ++q)
    for (int k = 0; k < 3; ++k) cen[k] += 2 * SES_CORNER[side[q]][k];
  /* m = (ma + mb)/2 - cen/ns, scaled by 2 ns to stay integral */
  for (int k = 0; k < 3; ++k) m[k] = (ma[k] + mb[k]) * ns - 2 * cen[k];
  const int *n = SES_FACE_N[f];
  dvec[0] = m[1] * n[2] - m[2] * n[1];
  dvec[1] = m[2] * n[0] - m[0] * n[2];
  dvec[2] = m[0] * n[1] - m[1] * n[0];
  const long dot = (mb[0] - ma[0]) * dvec[0] + (mb[1] - ma[1]) * dvec[1] + (mb[2] - ma[2]) * dvec[2];
  if (dot > 0)
    succ[ea] = eb;
  else
    succ[eb] = ea;
}

/* Loops of one cube case: up to 4 loops of up to 12 edges; returns the number of loops. */
static int case_loops(int cs, int loops[4][12], int len[4]) {
  int succ[12];
  for (int e = 0; e < 12; ++e) succ[e] = -1;
  for (int f = 0; f < 6; ++f) {
    const int *q = SES_FACE[f];
    int cross[4], nc = 0, ins[4], ni = 0;
    for (int s = 0; s < 4; ++s) {
      const int a = q[s], b = q[(s + 1) & 3];
      if (((cs >> a) & 1) != ((cs >> b) & 1)) cross[nc++] = s;
      if ((cs >> a) & 1) ins[ni++] = a;
    }
    if (nc == 2) {
      add_segment(f, edge_of(q[cross[0]], q[(cross[0] + 1) & 3]), edge_of(q[cross[1]], q[(cross[1] + 1) & 3]), ins,
                  ni, succ);
    } else if (nc == 4) {
      /* cut each inside corner off: join the two face edges that meet at it */
      for (int s = 0; s < 4; ++s) {
        const int c = q[s];
        if (!((cs >> c) & 1)) continue;
        add_segment(f, edge_of(q[(s + 3) & 3], c), edge_of(c, q[(s + 1) & 3]), &c, 1, succ);
      }
    }
  }
  int used[12] = {0}, n_loops = 0;
  for (int s = 0; s < 12; ++s) {
    if (succ[s] < 0 || used[s]) continue;
    int L = 0, cur = s;
    do {
      loops[n_loops][L++] = cur;
      used[cur] = 1;
      cur = succ[cur];
    } while (cur != s && cur >= 0 && L < 12);
    len[n_loops] = L;
    ++n_loops;
  }
  return n_loops;
}

/*
 * Marching cubes over the whole grid.  Writes at most max_tris triangles
 * (tris: [max_tris][3][3] world coordinates; edges: [max_tris][3] vertex
 * labels as above) and returns the total number of triangles.
 */
int64_t orc_ses_mc(const uint16_t *edt2, const int32_t *dims, const float *origin, float h, float probe,
                   const int32_t *offset, int64_t max_tris, double *tris, int64_t *edges) {
  const int64_t nx = dims[0], ny = dims[1], nz = dims[2];
  const int64_t o0 = offset ? offset[0] : 0, o1 = offset ? offset[1] : 0, o2 = offset ? offset[2] : 0;
  int64_t t = 0;
  for (int64_t k = 0; k + 1 < nz; ++k)
    for (int64_t j = 0; j + 1 < ny; ++j)
      for (int64_t i = 0; i + 1 < nx; ++i) {
        int cs = 0;
        double f[8], X[8][3];
        for (int c = 0; c < 8; ++c) {
          const int64_t a = i + SES_CORNER[c][0], b = j + SES_CORNER[c][1], d = k + SES_CORNER[c][2];
          const uint16_t e = edt2[(d * ny + b) * nx + a];
          if (ses_in(e, h, probe)) cs |= 1 << c;
          f[c] = sqrt((double)e) * (double)h - (double)probe;
          X[c][0] = (double)origin[0] + (double)h * (double)(a + o0);
          X[c][1] = (double)origin[1] + (double)h * (double)(b + o1);
          X[c][2] = (double)origin[2] + (double)h * (double)(d + o2);
        }
        if (cs == 0 || cs == 255) continue;
        int loops[4][12], len[4];
        const int nl = case_loops(cs, loops, len);
        const int64_t cell = (k * (ny - 1) + j) * (nx - 1) + i;
        for (int l = 0; l < nl; ++l) {
          double P[12][3], M[3] = {0.0, 0.0, 0.0};
          for (int q = 0; q < len[l]; ++q) {
            const int a = SES_EDGE[loops[l][q]][0], b = SES_EDGE[loops[l][q]][1];
            double s = f[a] == f[b] ? 0.5 : f[a] / (f[a] - f[b]);
            s = s < 0.0 ? 0.0 : (s > 1.0 ? 1.0 : s);
            for (int d = 0; d < 3; ++d) {
              P[q][d] = X[a][d] + s * (X[b][d] - X[a][d]);
              M[d] += P[q][d];
            }
          }
          for (int d = 0; d < 3; ++d) M[d] /= (double)len[l];
          const int n_t = len[l] == 3 ? 1 : len[l];
          for (int q = 0; q < n_t; ++q) {
            if (t < max_tris) {
              const double *V[3];
              int64_t lab[3];
              if (len[l] == 3) {
                for (int v = 0; v < 3; ++v) {
                  V[v] = P[v];
                  lab[v] = cell * 16 + loops[l][v];
                }
              } else {
                const int q1 = (q + 1) % len[l];
                V[0] = M;
                V[1] = P[q];
                V[2] = P[q1];
                lab[0] = cell * 16 + 12 + l;
                lab[1] = cell * 16 + loops[l][q];
                lab[2] = cell * 16 + loops[l][q1];
              }
              for (int v = 0; v < 3; ++v) {
                for (int d = 0; d < 3; ++d) tris[(t * 3 + v) * 3 + d] = V[v][d];
                if (edges) edges[t * 3 + v] = lab[v];
              }
            }
            ++t;
          }
        }
      }
  return t;
}

/* Number of triangles of every case (for pins on the case construction). */
void orc_ses_case_counts(int32_t *counts) {
  for (int cs = 0; cs < 256; ++cs) {
    int loops[4][12], len[4], n = 0;
    const int nl = (cs == 0 || cs == 255) ? 0 : case_loops(cs, loops, len);
    for (int l = 0; l < nl; ++l) n += len[l] == 3 ? 1 : len[l];
    counts[cs] = n;
  }
}
