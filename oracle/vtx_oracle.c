/*
 * vtx_oracle.c -- plain CPU FP64 oracle for the meshless molecular ray-caster.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * CPU-baseline leg of the benchmark load this library.  The CUDA renderer
 * never links, imports or calls it, and the two share no code: this file
 * defines its own camera record (same 64-byte layout, because both read the
 * same camera arrays) and re-derives every formula from the geometry.
 *
 * What it computes (the paper: Methods, "Meshless Representations" and
 * "High Quality Rendering"):
 *   - a molecule is a set of atoms with positions, radii and connectivity;
 *   - each primitive (a van der Waals sphere, or the capped cylinder of a
 *     bond in ball-and-stick) is drawn by ray-casting its implicit surface,
 *     so the visible surface at a pixel is the NEAREST ray/primitive hit;
 *   - lighting is deferred: shading runs on the per-pixel hit record and
 *     ambient occlusion is a screen-space pass over the depth buffer (the
 *     paper cites Mittring 2007 for it).
 * The paper gives no formulas, so the definitions below are the plain ones:
 * a brute-force loop over every (pixel, primitive) pair in FP64, a
 * Blinn-Phong "glossy" shade, a Crytek-style hemisphere SSAO and a sigmoid
 * soft-edge compositor.  Every constant the paper leaves open is an argument.
 *
 * Conventions.  View frame is right-handed: x = right, y = up, z toward the
 * viewer; the camera looks down -z.  View coordinates of a world point X are
 * (R.(X-E), U.(X-E), -F.(X-E)) with the float32 basis exactly as passed
 * (promoted to double, not re-normalised).  Pixel (px, py), row 0 at the top,
 * has its ray through the centre (px+0.5, py+0.5):
 *     a = (2(px+0.5)/W - 1) tan(fovy/2) W/H,  b = (1 - 2(py+0.5)/H) tan(fovy/2),
 *     u = (a, b, -1).
 * Because u_z = -1 the ray parameter t of a point t*u IS its depth.
 *
 * Numerics.  FP64 throughout, no fast-math, compiled with -ffp-contract=off
 * so that x86-64 and aarch64 round identically.  Ray/sphere uses the
 * closest-approach form (t_c = u.C/|u|^2, q = C - t_c u, rho^2 = |q|^2,
 * t = t_c - sqrt((r^2 - rho^2)/|u|^2)), which keeps r^2 - rho^2 accurate even
 * 36,000 A from the eye, where the textbook quadratic loses every digit.
 * Parity unpinned: the shading and SSAO constants (the paper names the
 * techniques, not their parameters).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef struct {
  float eye[3], forward[3], right[3], up[3];
  float tan_half_fovy, znear;
  int32_t width, height;
} orc_camera;

enum {
  ORC_FLAG_TIE = 1,    /* two nearest candidate depths closer than tie_tol */
  ORC_FLAG_GRAZE = 2,  /* a primitive boundary (silhouette, rim) passes within graze_tol in front */
  ORC_FLAG_NEAR = 4,   /* an entry point within graze_tol of the near plane */
  ORC_FLAG_SPLIT = 16, /* bond hit within graze_tol of the half-bond colour split */
  ORC_FLAG_GRID = 32,  /* an SSAO sample within grid_tol px of a pixel-grid line */
  ORC_FLAG_MARGIN = 64,/* an SSAO occlusion test within its error margin of the threshold */
  ORC_FLAG_FETCH = 128,/* an SSAO sample fetched a pixel whose visible surface is in doubt */
  ORC_FLAG_CUTOFF = 256, /* soft: a primitive within tol of the -4 px cutoff */
  ORC_FLAG_ORDER = 512,  /* soft: two contributors' centre depths within tol */
  ORC_FLAG_STOP = 1024,  /* soft: transmittance within tol of the stop threshold */
  ORC_FLAG_CLAMP = 2048, /* soft: opacity within tol of the 0.99 clamp */
  ORC_FLAG_BAND = 8192,  /* toon: diffuse term within tol of a band boundary */
  ORC_FLAG_EDGE = 16384  /* outline: a neighbour's depth step within tol of the threshold */
};

#define ORC_NO_ID 0xFFFFFFFFu

typedef struct {
  double E[3], R[3], U[3], F[3];
  double th, aspect, znear, f; /* f = H / (2 tan(fovy/2)): pixels per unit of image-plane slope */
  int W, H;
} ocam;

static void cam_load(const orc_camera *c, ocam *o) {
  for (int k = 0; k < 3; ++k) {
    o->E[k] = c->eye[k];
    o->R[k] = c->right[k];
    o->U[k] = c->up[k];
    o->F[k] = c->forward[k];
  }
  o->th = c->tan_half_fovy;
  o->W = c->width;
  o->H = c->height;
  o->aspect = (double)c->width / (double)c->height;
  o->znear = c->znear;
  o->f = (double)c->height / (2.0 * o->th);
}

static inline double dot3(const double *a, const double *b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }

static inline void cross3(const double *a, const double *b, double *o) {
  o[0] = a[1] * b[2] - a[2] * b[1];
  o[1] = a[2] * b[0] - a[0] * b[2];
  o[2] = a[0] * b[1] - a[1] * b[0];
}

/* View coordinates of a world point given as float32 (exactly promoted). */
static inline void to_view_f(const ocam *c, const float *X, double *V) {
  double d[3] = {(double)X[0] - c->E[0], (double)X[1] - c->E[1], (double)X[2] - c->E[2]};
  V[0] = dot3(c->R, d);
  V[1] = dot3(c->U, d);
  V[2] = -dot3(c->F, d);
}

static inline void to_view_d(const ocam *c, const double *X, double *V) {
  double d[3] = {X[0] - c->E[0], X[1] - c->E[1], X[2] - c->E[2]};
  V[0] = dot3(c->R, d);
  V[1] = dot3(c->U, d);
  V[2] = -dot3(c->F, d);
}

/* Ray direction of the pixel whose centre is at (px+0.5, py+0.5). */
static inline void pixel_ray(const ocam *c, int px, int py, double *u) {
  u[0] = (2.0 * (px + 0.5) / c->W - 1.0) * c->th * c->aspect;
  u[1] = (1.0 - 2.0 * (py + 0.5) / c->H) * c->th;
  u[2] = -1.0;
}

/* ---------------------------------------------------------------- hits -- */

typedef struct {
  double t1;     /* nearest accepted depth */
  uint32_t id1;  /* its primitive id (ties: smaller id) */
  double t2;     /* second nearest accepted depth among other primitives */
  double tg;     /* nearest depth at which some primitive boundary passes within graze_tol */
  int near;      /* some entry point within graze_tol of the near plane */
} hitstate;

static void hs_init(hitstate *s) {
  s->t1 = INFINITY;
  s->id1 = ORC_NO_ID;
  s->t2 = INFINITY;
  s->tg = INFINITY;
  s->near = 0;
}

static inline void hs_add(hitstate *s, double t, uint32_t id) {
  if (t < s->t1 || (t == s->t1 && id < s->id1)) {
    s->t2 = s->t1;
    s->t1 = t;
    s->id1 = id;
  } else if (t < s->t2) {
    s->t2 = t;
  }
}

static void hs_merge(hitstate *a, const hitstate *b) {
  if (b->id1 != ORC_NO_ID) {
    double bt2 = b->t2;
    hs_add(a, b->t1, b->id1);
    if (bt2 < a->t2) a->t2 = bt2;
  }
  if (b->tg < a->tg) a->tg = b->tg;
  a->near |= b->near;
}

/* Sphere with view-space centre C and radius r against ray u.
 * Returns 1 and the entry depth when the entry point exists; records boundary proximity. */
typedef struct {
  int hit;          /* 1: entry point exists at or beyond the near plane */
  double t;         /* entry depth */
  double amb_t;     /* depth of a boundary within graze_tol (INFINITY if none) */
  int near_amb;
} primhit;

static inline primhit sphere_hit(const double *C, double r, const double *u, double uu, double znear,
                                 double graze_tol) {
  primhit h = {0, INFINITY, INFINITY, 0};
  double tc = dot3(u, C) / uu;
  double q[3] = {C[0] - tc * u[0], C[1] - tc * u[1], C[2] - tc * u[2]};
  double rho2 = dot3(q, q);
  double dr = r * r - rho2;
  if (fabs(dr) < 2.0 * r * graze_tol && tc >= znear - graze_tol) h.amb_t = tc;
  if (dr < 0.0) return h;
  double t = tc - sqrt(dr / uu);
  if (fabs(t - znear) < graze_tol) h.near_amb = 1;
  if (t < znear) return h;
  h.hit = 1;
  h.t = t;
  return h;
}

/* Capped cylinder between view-space points Ci, Cj with radius rb.
 * Works relative to the midpoint M so that nothing cancels far from the eye.
 * Optional outputs: surface normal (view space) and axial coordinate of the hit. */
static inline primhit cylinder_hit(const double *Ci, const double *Cj, double rb, const double *u, double uu,
                                   double znear, double graze_tol, double *normal, double *axial, double *sil) {
  primhit h = {0, INFINITY, INFINITY, 0};
  double M[3] = {0.5 * (Ci[0] + Cj[0]), 0.5 * (Ci[1] + Cj[1]), 0.5 * (Ci[2] + Cj[2])};
  double Av[3] = {Cj[0] - Ci[0], Cj[1] - Ci[1], Cj[2] - Ci[2]};
  double L = sqrt(dot3(Av, Av));
  double A[3] = {Av[0] / L, Av[1] / L, Av[2] / L};
  double hl = 0.5 * L;
  double tM = dot3(u, M) / uu;
  double o[3] = {tM * u[0] - M[0], tM * u[1] - M[1], tM * u[2] - M[2]};
  double ua = dot3(u, A), oa = dot3(o, A);
  double up[3] = {u[0] - ua * A[0], u[1] - ua * A[1], u[2] - ua * A[2]};
  double op[3] = {o[0] - oa * A[0], o[1] - oa * A[1], o[2] - oa * A[2]};
  double a2 = dot3(up, up), b2 = dot3(op, up), c2 = dot3(op, op) - rb * rb;
  double best = INFINITY;
  int kind = 0; /* 1 side, 2 cap at +hl, 3 cap at -hl */
  double tol2 = 2.0 * rb * graze_tol;
  if (a2 > 1e-300) {
    double disc = b2 * b2 - a2 * c2;
    /* disc / a2 = rb^2 - (distance from the axis line to the ray)^2 */
    if (fabs(disc / a2) < tol2) {
      double s0 = -b2 / a2;
      double ax0 = oa + s0 * ua;
      if (fabs(ax0) <= hl + graze_tol && tM + s0 >= znear - graze_tol && tM + s0 < h.amb_t) h.amb_t = tM + s0;
    }
    if (disc >= 0.0) {
      double s1 = (-b2 - sqrt(disc)) / a2;
      double ax = oa + s1 * ua;
      if (fabs(fabs(ax) - hl) < graze_tol && tM + s1 >= znear - graze_tol && tM + s1 < h.amb_t) h.amb_t = tM + s1;
      if (fabs(ax) <= hl && s1 < best) {
        best = s1;
        kind = 1;
      }
    }
  }
  if (fabs(ua) > 1e-300) {
    for (int sgn = 0; sgn < 2; ++sgn) {
      double target = sgn == 0 ? hl : -hl;
      double s = (target - oa) / ua;
      double qv[3] = {op[0] + s * up[0], op[1] + s * up[1], op[2] + s * up[2]};
      double rad2 = dot3(qv, qv);
      if (fabs(rb * rb - rad2) < tol2 && tM + s >= znear - graze_tol && tM + s < h.amb_t) h.amb_t = tM + s;
      if (rad2 <= rb * rb && s < best) {
        best = s;
        kind = sgn == 0 ? 2 : 3;
      }
    }
  }
  if (kind == 0) return h;
  double t = tM + best;
  if (fabs(t - znear) < graze_tol) h.near_amb = 1;
  if (t < znear) return h;
  h.hit = 1;
  h.t = t;
  if (sil) {
    /* relative distance of the hit to the silhouette of the surface it lies on */
    if (kind == 1) {
      *sil = (b2 * b2 - a2 * c2) / a2 / (2.0 * rb * rb);
    } else {
      double qv[3] = {op[0] + best * up[0], op[1] + best * up[1], op[2] + best * up[2]};
      *sil = (rb * rb - dot3(qv, qv)) / (2.0 * rb * rb);
    }
  }
  if (normal) {
    if (kind == 1) {
      for (int k = 0; k < 3; ++k) normal[k] = (op[k] + best * up[k]) / rb;
    } else {
      double sg = kind == 2 ? 1.0 : -1.0;
      for (int k = 0; k < 3; ++k) normal[k] = sg * A[k];
    }
  }
  if (axial) *axial = oa + best * ua;
  return h;
}

/* Sphere radius per representation: 0 van der Waals (r), 1 ball-and-stick (ball radius),
 * 2 sticks (bond radius), 3 solvent accessible surface (r + probe, summed in float32 as stored). */
static inline double sphere_radius(int mode, float ball_radius, float bond_radius, float probe, const float *rec) {
  if (mode == 1) return (double)ball_radius;
  if (mode == 2) return (double)bond_radius;
  if (mode == 3) {
    float r = rec[3] + probe;
    return (double)r;
  }
  return (double)rec[3];
}

/* Clipping (Fig. 1C): an atom is kept when n.X + d >= 0; plane NULL or n = 0 keeps everything. */
static inline int clip_keep(const float *plane, const float *X) {
  if (!plane || (plane[0] == 0.0f && plane[1] == 0.0f && plane[2] == 0.0f)) return 1;
  double v = (double)plane[0] * X[0] + (double)plane[1] * X[1] + (double)plane[2] * X[2] + (double)plane[3];
  return v >= 0.0;
}

/*
 * Nearest hit at each listed pixel, brute force over every primitive.
 * pix: n_pix (px, py) pairs.  Primitive ids: atoms 0..n_atoms-1, then bonds
 * n_atoms + b (ball-and-stick mode only).
 * Outputs per pixel: depth (INFINITY for background), id (0xFFFFFFFF for
 * background), normal[3] (view space, 0 for background), gap = second minus
 * first depth, flags (ORC_FLAG_*), side (bonds: 0 when the hit lies on atom
 * i's half, 1 on atom j's; -1 otherwise), sil = (R^2 - rho^2) / (2 R^2): how
 * far, relative to the radius R of the surface hit, the ray passes inside
 * that surface's silhouette (rho: ray-to-centre or ray-to-axis distance).
 */
int orc_hits(const float *xyzr, int64_t n_atoms, const uint32_t *bonds, int64_t n_bonds, int32_t mode,
             float ball_radius, float bond_radius, float probe, const float *clip, const orc_camera *camera,
             const int32_t *pix, int64_t n_pix, double tie_tol, double graze_tol, double *depth, uint32_t *id,
             double *normal, double *gap, int32_t *flags, int32_t *side, double *sil, int32_t n_threads) {
  ocam c;
  cam_load(camera, &c);
  if (mode != 1 && mode != 2) n_bonds = 0;
  double *rays = (double *)malloc(sizeof(double) * 4 * (size_t)(n_pix > 0 ? n_pix : 1));
  for (int64_t p = 0; p < n_pix; ++p) {
    pixel_ray(&c, pix[2 * p], pix[2 * p + 1], rays + 4 * p);
    rays[4 * p + 3] = dot3(rays + 4 * p, rays + 4 * p);
  }
  int T = 1;
#ifdef _OPENMP
  T = n_threads > 0 ? n_threads : omp_get_max_threads();
#endif
  int64_t n_prims = n_atoms + n_bonds;
  if (n_prims < T) T = n_prims > 0 ? (int)n_prims : 1;
  hitstate *st = (hitstate *)malloc(sizeof(hitstate) * (size_t)T * (size_t)(n_pix > 0 ? n_pix : 1));
  const int64_t PB = 64;
#ifdef _OPENMP
#pragma omp parallel num_threads(T)
#endif
  {
    int tid = 0;
#ifdef _OPENMP
    tid = omp_get_thread_num();
#endif
    hitstate *my = st + (size_t)tid * (size_t)n_pix;
    for (int64_t p = 0; p < n_pix; ++p) hs_init(my + p);
    int64_t lo = n_prims * tid / T, hi = n_prims * (tid + 1) / T;
    for (int64_t p0 = 0; p0 < n_pix; p0 += PB) {
      int64_t p1 = p0 + PB < n_pix ? p0 + PB : n_pix;
      for (int64_t k = lo; k < hi; ++k) {
        if (k < n_atoms) {
          if (!clip_keep(clip, xyzr + 4 * k)) continue;
          double C[3];
          to_view_f(&c, xyzr + 4 * k, C);
          double r = sphere_radius(mode, ball_radius, bond_radius, probe, xyzr + 4 * k);
          for (int64_t p = p0; p < p1; ++p) {
            primhit h = sphere_hit(C, r, rays + 4 * p, rays[4 * p + 3], c.znear, graze_tol);
            if (h.amb_t < my[p].tg) my[p].tg = h.amb_t;
            my[p].near |= h.near_amb;
            if (h.hit) hs_add(my + p, h.t, (uint32_t)k);
          }
        } else {
          int64_t b = k - n_atoms;
          if (!clip_keep(clip, xyzr + 4 * (int64_t)bonds[2 * b]) || !clip_keep(clip, xyzr + 4 * (int64_t)bonds[2 * b + 1]))
            continue;
          double Ci[3], Cj[3];
          to_view_f(&c, xyzr + 4 * (int64_t)bonds[2 * b], Ci);
          to_view_f(&c, xyzr + 4 * (int64_t)bonds[2 * b + 1], Cj);
          for (int64_t p = p0; p < p1; ++p) {
            primhit h =
                cylinder_hit(Ci, Cj, bond_radius, rays + 4 * p, rays[4 * p + 3], c.znear, graze_tol, 0, 0, 0);
            if (h.amb_t < my[p].tg) my[p].tg = h.amb_t;
            my[p].near |= h.near_amb;
            if (h.hit) hs_add(my + p, h.t, (uint32_t)k);
          }
        }
      }
    }
  }
  for (int64_t p = 0; p < n_pix; ++p) {
    hitstate s;
    hs_init(&s);
    for (int t = 0; t < T; ++t) hs_merge(&s, st + (size_t)t * (size_t)n_pix + p);
    const double *u = rays + 4 * p;
    int fl = 0;
    if (s.t2 - s.t1 < tie_tol) fl |= ORC_FLAG_TIE;
    if (s.tg < INFINITY && s.tg <= s.t1 + tie_tol) fl |= ORC_FLAG_GRAZE;
    if (s.near) fl |= ORC_FLAG_NEAR;
    depth[p] = s.t1;
    id[p] = s.id1;
    gap[p] = s.t2 - s.t1;
    side[p] = -1;
    sil[p] = 0.0;
    normal[3 * p] = normal[3 * p + 1] = normal[3 * p + 2] = 0.0;
    if (s.id1 != ORC_NO_ID) {
      double P[3] = {s.t1 * u[0], s.t1 * u[1], s.t1 * u[2]};
      if ((int64_t)s.id1 < n_atoms) {
        double C[3];
        to_view_f(&c, xyzr + 4 * (int64_t)s.id1, C);
        double r = sphere_radius(mode, ball_radius, bond_radius, probe, xyzr + 4 * (int64_t)s.id1);
        for (int k = 0; k < 3; ++k) normal[3 * p + k] = (P[k] - C[k]) / r;
        double tc = dot3(u, C) / u[3];
        double q[3] = {C[0] - tc * u[0], C[1] - tc * u[1], C[2] - tc * u[2]};
        sil[p] = (r * r - dot3(q, q)) / (2.0 * r * r);
      } else {
        int64_t b = (int64_t)s.id1 - n_atoms;
        double Ci[3], Cj[3], nrm[3], ax = 0.0;
        to_view_f(&c, xyzr + 4 * (int64_t)bonds[2 * b], Ci);
        to_view_f(&c, xyzr + 4 * (int64_t)bonds[2 * b + 1], Cj);
        cylinder_hit(Ci, Cj, bond_radius, u, u[3], c.znear, graze_tol, nrm, &ax, sil + p);
        for (int k = 0; k < 3; ++k) normal[3 * p + k] = nrm[k];
        side[p] = ax <= 0.0 ? 0 : 1;
        if (fabs(ax) < graze_tol) fl |= ORC_FLAG_SPLIT;
      }
    }
    flags[p] = fl;
  }
  free(st);
  free(rays);
  return 0;
}

/* ------------------------------------------------------------- shading -- */

/*
 * Blinn-Phong ("glossy" in the paper's list of shading modes), directional
 * light L (view space, normalised here), viewer direction V = -u/|u|,
 * half vector H = (L+V)/|L+V|:
 *   rgb = clamp(albedo (ka + kd max(n.L,0)) + ks [n.L>0] max(n.H,0)^shininess, 0, 1).
 * Albedo is the element colour of the atom, or of the bond's atom on the hit
 * half.  Background pixels get the background colour.
 */
void orc_shade(const uint8_t *elem, const float *palette, int64_t n_atoms, const uint32_t *bonds,
               const orc_camera *camera, const int32_t *pix, int64_t n_pix, const uint32_t *id, const double *normal,
               const int32_t *side, const float *light_dir, double ka, double kd, double ks, double shininess,
               const float *background, int32_t model, int32_t toon_levels, double band_tol, double *rgb,
               int32_t *flags) {
  ocam c;
  cam_load(camera, &c);
  double L[3] = {light_dir[0], light_dir[1], light_dir[2]};
  double ln = sqrt(dot3(L, L));
  for (int k = 0; k < 3; ++k) L[k] /= ln;
  for (int64_t p = 0; p < n_pix; ++p) {
    if (id[p] == ORC_NO_ID) {
      for (int k = 0; k < 3; ++k) rgb[3 * p + k] = background[k];
      continue;
    }
    int64_t atom;
    if ((int64_t)id[p] < n_atoms)
      atom = id[p];
    else
      atom = bonds[2 * ((int64_t)id[p] - n_atoms) + (side[p] > 0 ? 1 : 0)];
    const float *alb = palette + 3 * (int)elem[atom];
    double u[3];
    pixel_ray(&c, pix[2 * p], pix[2 * p + 1], u);
    double un = sqrt(dot3(u, u));
    double V[3] = {-u[0] / un, -u[1] / un, -u[2] / un};
    double Hh[3] = {L[0] + V[0], L[1] + V[1], L[2] + V[2]};
    double hn = sqrt(dot3(Hh, Hh));
    for (int k = 0; k < 3; ++k) Hh[k] /= hn;
    const double *n = normal + 3 * p;
    double nl = dot3(n, L), nh = dot3(n, Hh);
    double d = nl > 0.0 ? nl : 0.0;
    double diff = ka + kd * d, spec = 0.0;
    if (model == 0) {
      spec = nl > 0.0 ? ks * pow(nh > 0.0 ? nh : 0.0, shininess) : 0.0;
    } else if (model == 1) {
      diff = 1.0;
    } else if (model == 3) {
      double x = d * toon_levels;
      double band = floor(x);
      if (band > toon_levels - 1) band = toon_levels - 1;
      if (fabs(x - floor(x + 0.5)) < band_tol && x > 0.5 && x < toon_levels - 0.5) flags[p] |= ORC_FLAG_BAND;
      diff = ka + kd * band / (toon_levels - 1);
    }
    for (int k = 0; k < 3; ++k) {
      double v = (double)alb[k] * diff + spec;
      rgb[3 * p + k] = v < 0.0 ? 0.0 : (v > 1.0 ? 1.0 : v);
    }
  }
}

/* ---------------------------------------------------------------- SSAO -- */

/*
 * Screen-space ambient occlusion, step 1: sample positions.
 * For a covered pixel with hit point P = t u and normal n, the tangent frame
 * is T = normalize(n x a) with a = (0,1,0), or (1,0,0) when |n_y| > 0.9, and
 * B = n x T.  Sample j is S_j = P + radius (k_x T + k_y B + k_z n), projected
 * to pixel coordinates and floored.  Output per (pixel, sample): the fetched
 * pixel (fx, fy) or (-1, -1) when off screen, and the sample's own depth.
 *
 * Ambiguity band (a test tolerance, not part of the method): a renderer that
 * computes the hit point in FP32 places the sample slightly off S_j, so a
 * sample that projects within `band` px of a pixel-grid line may be floored
 * to the neighbouring pixel; such a pixel is flagged ORC_FLAG_GRID.  Per axis
 *   band = grid_abs + grid_rel |off| + (f / ds) err_pos[p] + |off| err_t[p] / ds,
 * where off is the sample's offset from the pixel centre (px), ds its depth,
 * and err_pos / err_t (per pixel, inputs) bound the error of the sample's
 * position (A) and of the hit depth.
 */
void orc_ssao_project(const orc_camera *camera, const int32_t *pix, int64_t n_pix, const double *depth,
                      const uint32_t *id, const double *normal, const float *kernel, int32_t n_samples,
                      double radius, double grid_abs, double grid_rel, const double *err_pos, const double *err_t,
                      int32_t *fetch, double *sample_depth, int32_t *flags) {
  ocam c;
  cam_load(camera, &c);
  for (int64_t p = 0; p < n_pix; ++p) {
    for (int j = 0; j < n_samples; ++j) {
      fetch[2 * (p * n_samples + j)] = -1;
      fetch[2 * (p * n_samples + j) + 1] = -1;
      sample_depth[p * n_samples + j] = INFINITY;
    }
    if (id[p] == ORC_NO_ID) continue;
    double u[3];
    pixel_ray(&c, pix[2 * p], pix[2 * p + 1], u);
    double P[3] = {depth[p] * u[0], depth[p] * u[1], depth[p] * u[2]};
    const double *n = normal + 3 * p;
    double a[3] = {0.0, 1.0, 0.0};
    if (fabs(n[1]) > 0.9) {
      a[0] = 1.0;
      a[1] = 0.0;
    }
    double Tv[3], Bv[3];
    cross3(n, a, Tv);
    double tn = sqrt(dot3(Tv, Tv));
    for (int k = 0; k < 3; ++k) Tv[k] /= tn;
    cross3(n, Tv, Bv);
    for (int j = 0; j < n_samples; ++j) {
      const float *kj = kernel + 3 * j;
      double S[3];
      for (int k = 0; k < 3; ++k) S[k] = P[k] + radius * (kj[0] * Tv[k] + kj[1] * Bv[k] + kj[2] * n[k]);
      double ds = -S[2];
      sample_depth[p * n_samples + j] = ds;
      if (ds <= 0.0) continue;
      double x = 0.5 * c.W * (1.0 + (S[0] / ds) / (c.th * c.aspect));
      double y = 0.5 * c.H * (1.0 - (S[1] / ds) / c.th);
      const double fd = c.f / ds;
      const double offx = x - (pix[2 * p] + 0.5), offy = y - (pix[2 * p + 1] + 0.5);
      const double bx = grid_abs + grid_rel * fabs(offx) + fd * err_pos[p] + fabs(offx) * err_t[p] / ds;
      const double by = grid_abs + grid_rel * fabs(offy) + fd * err_pos[p] + fabs(offy) * err_t[p] / ds;
      if (fabs(x - floor(x + 0.5)) < bx || fabs(y - floor(y + 0.5)) < by) flags[p] |= ORC_FLAG_GRID;
      double fx = floor(x), fy = floor(y);
      if (fx < 0.0 || fy < 0.0 || fx >= c.W || fy >= c.H) continue;
      fetch[2 * (p * n_samples + j)] = (int32_t)fx;
      fetch[2 * (p * n_samples + j) + 1] = (int32_t)fy;
    }
  }
}

/*
 * SSAO step 2: occlusion.  fetched_depth[p*ns+j] is the depth stored at the
 * fetched pixel (INFINITY for background or off screen).  A sample is
 * occluded when z_f <= depth(S_j) - bias; its weight is min(1, radius/|t - z_f|).
 * AO = 1 - (1/ns) sum occ_j w_j; background pixels get AO = 1.
 *
 * Ambiguity bands (test tolerances): fetched_amb[p*ns+j] holds the fetched
 * pixel's id flags, fetched_gap its second-minus-first depth and fetched_err
 * the bound on its depth error.  A fetched pixel whose visible surface is in
 * doubt (GRAZE or NEAR) flags ORC_FLAG_FETCH; a tie (TIE) can only move its
 * depth by its gap, which widens the occlusion margin.  An occlusion test
 * within
 *   margin = margin_abs + err_t[p] + fetched_err + err_pos[p] + 2e-7 |t - z_f|
 *            (+ fetched_gap for a tie)
 * of its threshold flags ORC_FLAG_MARGIN.
 */
void orc_ssao_resolve(int64_t n_pix, int32_t n_samples, const double *depth, const uint32_t *id,
                      const double *sample_depth, const double *fetched_depth, const int32_t *fetched_amb,
                      const double *fetched_gap, const double *fetched_err, double radius, double bias,
                      double margin_abs, const double *err_pos, const double *err_t, double *ao, int32_t *flags) {
  for (int64_t p = 0; p < n_pix; ++p) {
    if (id[p] == ORC_NO_ID) {
      ao[p] = 1.0;
      continue;
    }
    double occ = 0.0;
    for (int j = 0; j < n_samples; ++j) {
      const int64_t q = p * n_samples + j;
      double zf = fetched_depth[q];
      if (fetched_amb[q] & (ORC_FLAG_GRAZE | ORC_FLAG_NEAR)) flags[p] |= ORC_FLAG_FETCH;
      if (!(zf < INFINITY)) continue;
      double thr = sample_depth[q] - bias;
      double margin = margin_abs + err_t[p] + fetched_err[q] + err_pos[p] + 2e-7 * fabs(depth[p] - zf);
      if (fetched_amb[q] & ORC_FLAG_TIE) margin += fetched_gap[q];
      if (fabs(zf - thr) < margin) flags[p] |= ORC_FLAG_MARGIN;
      if (zf <= thr) {
        double dz = fabs(depth[p] - zf);
        double w = dz <= radius ? 1.0 : radius / dz;
        occ += w;
      }
    }
    ao[p] = 1.0 - occ / n_samples;
  }
}

/* -------------------------------------------------------- post-process -- */

/*
 * Outline and fog, after shading and ambient occlusion (colour in rgb, in
 * place).  nbr_depth[p*4 + u] is the depth at the 4-neighbour u (left, right,
 * up, down; INFINITY for background; NAN when outside the image, which is
 * ignored); nbr_amb marks id-ambiguous neighbours.  A step within edge_abs +
 * edge_rel * depth of the threshold flags the pixel (EDGE).  A covered pixel with a
 * neighbour that is background or deeper by more than outline_depth takes
 * outline_color.  Fog: f = density * clamp((t - near)/(far - near), 0, 1),
 * colour = (1 - f) colour + f background.
 */
void orc_post(int64_t n_pix, const double *depth, const uint32_t *id, const double *nbr_depth, const int32_t *nbr_amb,
              double outline_depth, const float *outline_color, double fog_near, double fog_far, double fog_density,
              const float *background, double edge_abs, double edge_rel, double *rgb, int32_t *flags) {
  for (int64_t p = 0; p < n_pix; ++p) {
    if (id[p] == ORC_NO_ID) continue;
    if (outline_depth > 0.0) {
      int edge = 0;
      for (int u = 0; u < 4; ++u) {
        double zq = nbr_depth[4 * p + u];
        if (zq != zq) continue;
        if (nbr_amb[4 * p + u]) flags[p] |= ORC_FLAG_FETCH;
        if (!(zq < INFINITY)) {
          edge = 1;
          continue;
        }
        double step = zq - depth[p];
        if (fabs(step - outline_depth) < edge_abs + edge_rel * depth[p]) flags[p] |= ORC_FLAG_EDGE;
        if (step > outline_depth) edge = 1;
      }
      if (edge)
        for (int k = 0; k < 3; ++k) rgb[3 * p + k] = outline_color[k];
    }
    if (fog_density > 0.0) {
      double span = fog_far - fog_near, fz;
      if (span > 0.0) {
        fz = (depth[p] - fog_near) / span;
        fz = fz < 0.0 ? 0.0 : (fz > 1.0 ? 1.0 : fz);
      } else {
        fz = depth[p] >= fog_far ? 1.0 : 0.0;
      }
      double fw = fog_density * fz;
      for (int k = 0; k < 3; ++k) rgb[3 * p + k] = rgb[3 * p + k] + fw * ((double)background[k] - rgb[3 * p + k]);
    }
  }
}

/* ---------------------------------------------------------- soft edges -- */

/*
 * Soft-edge sphere renderer (differentiable form).  Per pixel ray u and
 * sphere (view centre C, depth z_c = -C_z, radius r):
 *   t_c = u.C/|u|^2,  q = C - t_c u,  rho^2 = |q|^2         (distance to the ray)
 *   delta = (r - sqrt(rho^2 + 1e-12)) f / z_c                (signed px to silhouette)
 *   alpha = min(0.99, 1/(1 + exp(-delta/sigma)))
 *   g = sqrt(max(r^2 - rho^2, 0) + eta^2) - eta, eta = 0.05 r
 *   t_i = t_c - g/|u|   (smoothed entry depth),  n_i = (t_i u - C)/r
 * Contributors: z_c > near and delta >= -4, ordered by z_c then id.
 * Composite front to back: T_0 = 1, w_i = alpha_i T_i, T_{i+1} = T_i (1-alpha_i),
 * stop before i once T_i < 1e-4.  A = sum w_i, D = sum w_i t_i, N = sum w_i n_i.
 */
typedef struct {
  double zc, tc, rho2, delta, r;
  double C[3], q[3];
  int64_t i;
} softc;

static int softc_cmp(const void *a, const void *b) {
  const softc *x = (const softc *)a, *y = (const softc *)b;
  if (x->zc < y->zc) return -1;
  if (x->zc > y->zc) return 1;
  return x->i < y->i ? -1 : (x->i > y->i ? 1 : 0);
}

#define SOFT_CUTOFF (-4.0)
#define SOFT_TSTOP 1e-4
#define SOFT_AMAX 0.99

static int soft_collect(const ocam *c, const double *xyzr, int64_t n, const double *u, double uu, softc *buf,
                        int *fl, double tol) {
  int m = 0;
  for (int64_t i = 0; i < n; ++i) {
    double C[3];
    to_view_d(c, xyzr + 4 * i, C);
    double zc = -C[2];
    if (zc <= c->znear) continue;
    double r = xyzr[4 * i + 3];
    double tc = dot3(u, C) / uu;
    double q[3] = {C[0] - tc * u[0], C[1] - tc * u[1], C[2] - tc * u[2]};
    double rho2 = dot3(q, q);
    double delta = (r - sqrt(rho2 + 1e-12)) * c->f / zc;
    if (fabs(delta - SOFT_CUTOFF) < tol) *fl |= ORC_FLAG_CUTOFF;
    if (delta < SOFT_CUTOFF) continue;
    softc *s = buf + m++;
    s->zc = zc;
    s->tc = tc;
    s->rho2 = rho2;
    s->delta = delta;
    s->r = r;
    s->i = i;
    for (int k = 0; k < 3; ++k) {
      s->C[k] = C[k];
      s->q[k] = q[k];
    }
  }
  qsort(buf, (size_t)m, sizeof(softc), softc_cmp);
  for (int k = 1; k < m; ++k)
    if (buf[k].zc - buf[k - 1].zc < tol) *fl |= ORC_FLAG_ORDER;
  return m;
}

typedef struct {
  double alpha, sg, t, n[3], T, g, sq, m;
} softv;

static void soft_eval(const softc *s, const double *u, double uu, double sigma, softv *v) {
  double sg = 1.0 / (1.0 + exp(-s->delta / sigma));
  v->sg = sg;
  v->alpha = sg < SOFT_AMAX ? sg : SOFT_AMAX;
  double eta = 0.05 * s->r;
  double m = s->r * s->r - s->rho2;
  if (m < 0.0) m = 0.0;
  v->m = m;
  v->sq = sqrt(m + eta * eta);
  v->g = v->sq - eta;
  v->t = s->tc - v->g / sqrt(uu);
  for (int k = 0; k < 3; ++k) v->n[k] = (v->t * u[k] - s->C[k]) / s->r;
}

void orc_soft_forward(const double *xyzr, int64_t n, const orc_camera *camera, double sigma, const int32_t *pix,
                      int64_t n_pix, double amb_tol, double *A, double *D, double *N3, int32_t *n_used,
                      double *T_final, int32_t *flags, int32_t n_threads) {
  ocam c;
  cam_load(camera, &c);
  int T = 1;
#ifdef _OPENMP
  T = n_threads > 0 ? n_threads : omp_get_max_threads();
#endif
#ifdef _OPENMP
#pragma omp parallel num_threads(T)
#endif
  {
    softc *buf = (softc *)malloc(sizeof(softc) * (size_t)(n > 0 ? n : 1));
    softv v;
#ifdef _OPENMP
#pragma omp for schedule(dynamic, 16)
#endif
    for (int64_t p = 0; p < n_pix; ++p) {
      double u[3];
      pixel_ray(&c, pix[2 * p], pix[2 * p + 1], u);
      double uu = dot3(u, u);
      int fl = 0;
      int m = soft_collect(&c, xyzr, n, u, uu, buf, &fl, amb_tol);
      double Tr = 1.0, a = 0.0, d = 0.0, nn[3] = {0.0, 0.0, 0.0};
      int used = 0;
      for (int k = 0; k < m; ++k) {
        if (fabs(Tr - SOFT_TSTOP) < amb_tol * SOFT_TSTOP) fl |= ORC_FLAG_STOP;
        if (Tr < SOFT_TSTOP) break;
        soft_eval(buf + k, u, uu, sigma, &v);
        if (fabs(v.sg - SOFT_AMAX) < amb_tol) fl |= ORC_FLAG_CLAMP;
        double w = v.alpha * Tr;
        a += w;
        d += w * v.t;
        for (int j = 0; j < 3; ++j) nn[j] += w * v.n[j];
        Tr *= 1.0 - v.alpha;
        ++used;
      }
      A[p] = a;
      D[p] = d;
      for (int j = 0; j < 3; ++j) N3[3 * p + j] = nn[j];
      n_used[p] = used;
      T_final[p] = Tr;
      flags[p] = fl;
    }
    free(buf);
  }
}

/*
 * Vector-Jacobian product of the soft renderer: grad += d/d(x,y,z,r) of
 *   sum_p gA[p] A[p] + gD[p] D[p] + gN[p].N[p]
 * over the listed pixels.  Back to front with the division-free carry
 * R_i = alpha_{i+1} c_{i+1} + (1 - alpha_{i+1}) R_{i+1}, c_i = gA + gD t_i + gN.n_i,
 * so that dO/dalpha_i = T_i (c_i - R_i).  The stop index, the -4 px cutoff
 * and the 0.99 clamp are piecewise constant (zero derivative).
 */
void orc_soft_vjp(const double *xyzr, int64_t n, const orc_camera *camera, double sigma, const int32_t *pix,
                  int64_t n_pix, const double *gA, const double *gD, const double *gN, double *grad,
                  int32_t n_threads) {
  ocam c;
  cam_load(camera, &c);
  int T = 1;
#ifdef _OPENMP
  T = n_threads > 0 ? n_threads : omp_get_max_threads();
#endif
  double *acc = (double *)calloc((size_t)T * (size_t)(n > 0 ? n : 1) * 4, sizeof(double));
#ifdef _OPENMP
#pragma omp parallel num_threads(T)
#endif
  {
    int tid = 0;
#ifdef _OPENMP
    tid = omp_get_thread_num();
#endif
    double *g = acc + (size_t)tid * (size_t)n * 4;
    softc *buf = (softc *)malloc(sizeof(softc) * (size_t)(n > 0 ? n : 1));
    softv *vals = (softv *)malloc(sizeof(softv) * (size_t)(n > 0 ? n : 1));
#ifdef _OPENMP
#pragma omp for schedule(dynamic, 16)
#endif
    for (int64_t p = 0; p < n_pix; ++p) {
      if (gA[p] == 0.0 && gD[p] == 0.0 && gN[3 * p] == 0.0 && gN[3 * p + 1] == 0.0 && gN[3 * p + 2] == 0.0)
        continue;
      double u[3];
      pixel_ray(&c, pix[2 * p], pix[2 * p + 1], u);
      double uu = dot3(u, u), un = sqrt(uu);
      int fl = 0;
      int m = soft_collect(&c, xyzr, n, u, uu, buf, &fl, 0.0);
      double Tr = 1.0;
      int used = 0;
      for (int k = 0; k < m; ++k) {
        if (Tr < SOFT_TSTOP) break;
        soft_eval(buf + k, u, uu, sigma, vals + k);
        vals[k].T = Tr;
        Tr *= 1.0 - vals[k].alpha;
        ++used;
      }
      const double *gn = gN + 3 * p;
      double R = 0.0;
      for (int k = used - 1; k >= 0; --k) {
        const softc *s = buf + k;
        const softv *v = vals + k;
        double ci = gA[p] + gD[p] * v->t + dot3(gn, v->n);
        double w = v->alpha * v->T;
        double dalpha = v->T * (ci - R);
        R = v->alpha * ci + (1.0 - v->alpha) * R;
        /* alpha(delta) */
        double da_dd = v->sg < SOFT_AMAX ? v->sg * (1.0 - v->sg) / sigma : 0.0;
        double ddelta = dalpha * da_dd;
        double sq = sqrt(s->rho2 + 1e-12);
        double gC[3], gr;
        for (int j = 0; j < 3; ++j) gC[j] = -ddelta * (c.f / s->zc) * s->q[j] / sq;
        gC[2] += ddelta * s->delta / s->zc;
        gr = ddelta * c.f / s->zc;
        /* t_i(C, r) */
        double dg_drho2 = 0.0, dg_dr = 0.0;
        if (v->m > 0.0) {
          double eta = 0.05 * s->r;
          dg_drho2 = -0.5 / v->sq;
          dg_dr = (s->r + 0.05 * eta) / v->sq - 0.05;
        }
        double dt_dC[3];
        for (int j = 0; j < 3; ++j) dt_dC[j] = u[j] / uu - dg_drho2 * 2.0 * s->q[j] / un;
        double dt_dr = -dg_dr / un;
        /* upstream of t_i: w gD; of n_i: w gN; n_i = (t_i u - C)/r */
        double ut = w * gD[p];
        double ugn = w * dot3(u, gn);
        for (int j = 0; j < 3; ++j) gC[j] += ut * dt_dC[j] + (dt_dC[j] * ugn - w * gn[j]) / s->r;
        gr += ut * dt_dr + (ugn * dt_dr - w * dot3(gn, v->n)) / s->r;
        /* view -> world: C = (R.d, U.d, -F.d) */
        double *gi = g + 4 * s->i;
        for (int j = 0; j < 3; ++j) gi[j] += c.R[j] * gC[0] + c.U[j] * gC[1] - c.F[j] * gC[2];
        gi[3] += gr;
      }
    }
    free(buf);
    free(vals);
  }
  for (int t = 0; t < T; ++t)
    for (int64_t i = 0; i < 4 * n; ++i) grad[i] += acc[(size_t)t * (size_t)n * 4 + (size_t)i];
  free(acc);
}

int orc_abi_version(void) { return 1; }
