// vtx_device.cuh -- device-side math of the meshless ray-caster (sm_103a).
//
// Every primitive the paper draws without a mesh (Methods, "Meshless
// Representations": spheres for van der Waals / ball-and-stick atoms,
// cylinders for bonds) is ray-cast against its implicit surface.  Doing that
// in FP32 directly fails far from the eye: at 36,000 A an FP32 ulp is
// 4e-3 A, which flips silhouette pixels and ruins normals.  So each
// primitive gets a PRECISE SETUP in double-float arithmetic (pairs of FP32
// numbers; TwoSum after Knuth, TwoProduct via FMA after Dekker 1971): its
// projected reference point (u0, v0) in pixels, its reference depth and a
// 32-bit fixed-point depth key.  Per pixel the ray is then expressed
// relative to the primitive (every FP32 quantity is Angstrom-scale), which
// keeps depth and normal errors near 1e-7 A.  FP64 is avoided: GB300 runs it
// at a small fraction of its FP32 rate.
//
// Frames: the INTERNAL view frame used by the kernels is x right, y up,
// z = depth (forward); pixel rays are u = (a, b, 1).  Reported normals are
// in the right-handed view frame (x right, y up, z toward the viewer), i.e.
// the internal normal with z negated.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace vtx {

constexpr uint32_t kNoId = 0xFFFFFFFFu;
constexpr unsigned long long kBgKey = ~0ull;
constexpr long long kKeySpan = 4294966784LL;  // 2^32 - 512: object keys stay below the background key
constexpr float kKeySpanF = 4294966784.0f;
constexpr int kMaxViews = 16;
constexpr int kMaxSsao = 64;
constexpr int kMaxElem = 32;

// ------------------------------------------------------------ parameters --

// Per-camera constants, computed on the host in FP64 and stored as FP32.
struct ViewParams {
  float eye[3];
  float R[3], U[3], F[3];  // right, up, forward exactly as passed
  float f;                 // H / (2 tan_half_fovy): pixels per unit slope (FP32 rounding)
  float f_hi, f_lo;        // f as a double-float
  float inv_f;
  float cx, cy;            // W/2, H/2
  float znear;
  float pad0;
  // constants of the streaming cull test (cull_lean)
  float hc;                // f * (1 + 4e-6): pixels per slope, inflated by the test's relative rounding
  float e0;                // absolute pixel margin: 1e-4 + 1e-6 * (W + H)
  float cxm, cym;          // cx - 0.5, cy - 0.5
  float wm1, hm1;          // W - 1, H - 1
};

// Launch-wide geometry shared by every stage of a frame or batch.
struct Geometry {
  ViewParams views[kMaxViews];
  int n_views, n_frames, n_img;
  int W, H;
  int tile_w, tile_h, tiles_x, tiles_y, tiles_per_img;
  int mode;              // 0 vdW, 1 ball-and-stick, 2 sticks, 3 SAS
  float ball_radius, bond_radius;
  float probe;           // SAS probe radius
  float clip[4];         // clip plane (n, d); clip_on = n != 0
  int clip_on;
  int splat_max;         // max candidate pixels for the direct splat path
  int dbg_first_wait;    // test hook: polls allowed for the multi-view cull's first stage wait (-1: normal limit)
  int soft;              // 1 = soft-edge binning (dilated bounds, no splat, every survivor binned)
  int occl;              // 1 = occlusion pass allowed: survivors proven hidden by FP32 depth bounds skip setup
  float sigma;           // soft: sigmoid width in pixels
  long long stride;      // atom records per frame slot
  long long n_atoms;     // atoms of frame 0 (single frame) -- primitive ids of bonds start here
  long long n_bonds;
  long long surv_cap;    // survivor slots per image
  long long pix_per_img;
};

struct ShadeParams {
  int model;             // 0 glossy, 1 flat, 2 matte, 3 toon
  int toon_levels;
  float fog_near, fog_far, fog_density;
  float outline_depth;
  float outline_color[3];
  float ka, kd, ks, shin;
  float L[3];            // normalised light direction (right-handed view frame)
  float bg[3];
  float palette[kMaxElem][3];
  int n_elem;
  int ssao_n;
  float ssao_radius, ssao_bias;
  float kernel[kMaxSsao][3];
};

// Per-image mutable state (device memory).
struct ImageState {
  unsigned int zlo_bits;  // atomicMin of max(z - R, 0) over survivors (float bits)
  unsigned int zhi_bits;  // atomicMax of z + R over survivors
  unsigned int n_surv;    // survivors appended (may exceed the capacity)
  unsigned int valid;     // set by finalize when there is at least one survivor
  float zlo, S, invS;     // key = (depth - zlo) * S
  unsigned int occl;      // 1: this image runs the occlusion pass (many survivors per pixel)
  unsigned int n_vis;     // occlusion pass: survivors its test could not prove hidden (the kept list)
};

// Launch-wide status (device memory, read back by the host).
struct Status {
  unsigned int n_rec;           // binned records requested
  unsigned int overflow;        // bit 1 records, 2 entries, 4 a bounded wait gave up,
                                // 5 a decoded primitive id out of range
  unsigned long long n_entries; // binned (tile, primitive) entries requested
  unsigned int max_list;        // longest tile list seen by the raster stage
  unsigned int n_list;          // non-empty tiles listed by the scan (raster work list)
  unsigned int n_cov;           // covered pixels listed by the resolve's list pass
  unsigned int pad;
  unsigned long long n_terms;   // soft forward: sigmoid terms composited (sum over pixels)
  unsigned int soft_next;       // soft passes: the next entry of the non-empty tile list to take
  unsigned int tile_next;       // hard raster: the next entry of the non-empty tile list to take
};

// A binned primitive staged through shared memory (64 bytes).  Its tile box
// lives in a separate array (only the scatter stage reads it).
struct __align__(16) PrimRec {
  float u0h, u0l, v0h, v0l;  // projected reference point (pixels), double-float
  float zr, k, dz, rad;      // reference depth, A per pixel at zr, zr - centre depth, radius
  uint32_t key_lo;           // depth key of zr, low word (soft: centre-depth sort key)
  int key_hi;                // depth key of zr, high word (the key may leave [0, 2^32) for near-eye primitives)
  uint32_t id;               // primitive id
  float hl;                  // cylinder half length; 0 for spheres
  float ax, ay, az, pad;     // cylinder axis (internal frame)
};

// Sphere radius of an atom record in the current representation.
__device__ __forceinline__ float atom_radius(const Geometry &g, float w) {
  switch (g.mode) {
    case 1: return g.ball_radius;
    case 2: return g.bond_radius;
    case 3: return w + g.probe;
    default: return w;
  }
}

// Clipping (per atom centre): false when the atom is removed.
__device__ __forceinline__ bool clip_keep(const Geometry &g, float x, float y, float z) {
  return !g.clip_on || fmaf(g.clip[0], x, fmaf(g.clip[1], y, fmaf(g.clip[2], z, g.clip[3]))) >= 0.0f;
}

__device__ __forceinline__ long long rec_key(const PrimRec &p) {
  return (long long)(((unsigned long long)(unsigned)p.key_hi << 32) | (unsigned long long)p.key_lo);
}

// ------------------------------------------------------ double-float ops --
// Knuth TwoSum and Dekker/FMA TwoProduct; explicit round-to-nearest
// intrinsics keep the compiler from fusing or reassociating them.

struct df {
  float hi, lo;
};

__device__ __forceinline__ df two_sum(float a, float b) {
  float s = __fadd_rn(a, b);
  float bb = __fsub_rn(s, a);
  float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return {s, e};
}

__device__ __forceinline__ df df_norm(float hi, float lo) { return two_sum(hi, lo); }

__device__ __forceinline__ df df_add(df a, df b) {
  df s = two_sum(a.hi, b.hi);
  return df_norm(s.hi, __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo)));
}

__device__ __forceinline__ df df_add_f(df a, float b) {
  df s = two_sum(a.hi, b);
  return df_norm(s.hi, __fadd_rn(s.lo, a.lo));
}

__device__ __forceinline__ df df_neg(df a) { return {-a.hi, -a.lo}; }

__device__ __forceinline__ df df_mul_f(df a, float b) {
  float p = __fmul_rn(a.hi, b);
  float e = __fmaf_rn(a.hi, b, -p);
  e = __fmaf_rn(a.lo, b, e);
  return df_norm(p, e);
}

__device__ __forceinline__ df df_mul(df a, df b) {
  float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  return df_norm(p, e);
}

// a / b.  The first quotient only needs ~23 correct bits: the remainder
// a - q1 b is formed exactly (FMA TwoProduct) and its quotient corrects q1,
// leaving a relative error near 2^-44, so a reciprocal multiply suffices.
__device__ __forceinline__ df df_div(df a, df b) {
  const float rb = __frcp_rn(b.hi);
  float q1 = __fmul_rn(a.hi, rb);
  df r = df_add(a, df_neg(df_mul_f(b, q1)));
  float q2 = __fmul_rn(r.hi, rb);
  return df_norm(q1, q2);
}

__device__ __forceinline__ df df_dot3(const float *w, df x, df y, df z) {
  return df_add(df_add(df_mul_f(x, w[0]), df_mul_f(y, w[1])), df_mul_f(z, w[2]));
}

// Dekker's FastTwoSum: exact when |a| >= |b| (otherwise still a faithful sum
// whose error is below ulp(b), which is all the callers need).
__device__ __forceinline__ df fast_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  return {s, __fsub_rn(b, __fsub_rn(s, a))};
}

// w . (x, y, z) for FP32 weights and double-float operands: the three products
// of the high parts are exact (FMA TwoProduct), two TwoSums add them, and every
// rounding error plus the low-part products are summed in FP32.  Absolute
// error ~2^-46 of the largest product.
__device__ __forceinline__ df df_dot3_lean(const float *w, df x, df y, df z) {
  const float p0 = __fmul_rn(w[0], x.hi), p1 = __fmul_rn(w[1], y.hi), p2 = __fmul_rn(w[2], z.hi);
  float e = __fmaf_rn(w[0], x.hi, -p0);
  e = __fadd_rn(e, __fmaf_rn(w[1], y.hi, -p1));
  e = __fadd_rn(e, __fmaf_rn(w[2], z.hi, -p2));
  const df s01 = two_sum(p0, p1);
  const df s = two_sum(s01.hi, p2);
  e = __fadd_rn(e, __fadd_rn(s01.lo, s.lo));
  e = __fmaf_rn(w[0], x.lo, e);
  e = __fmaf_rn(w[1], y.lo, e);
  e = __fmaf_rn(w[2], z.lo, e);
  return fast_two_sum(s.hi, e);
}

// a / b with one exact remainder: q1 = a.hi / b.hi (to ~1 ulp), r = a - q1 b
// where q1 * b.hi is split exactly by an FMA (a.hi - p is exact, Sterbenz),
// then q = q1 + r / b.hi.  Relative error ~2^-44.
__device__ __forceinline__ df df_div_lean(df a, df b) {
  const float rb = __frcp_rn(b.hi);
  const float q1 = __fmul_rn(a.hi, rb);
  const float p = __fmul_rn(q1, b.hi);
  const float pe = __fmaf_rn(q1, b.hi, -p);
  float r = __fsub_rn(a.hi, p);
  r = __fsub_rn(r, pe);
  r = __fadd_rn(r, a.lo);
  r = __fmaf_rn(-q1, b.lo, r);
  return fast_two_sum(q1, __fmul_rn(r, rb));
}

__device__ __forceinline__ df df_mul_lean(df a, df b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  return fast_two_sum(p, e);
}

// ------------------------------------------------------------ per pixel --

struct PixRay {
  float pxc, pyc;  // pixel-centre coordinates (px + 0.5, py + 0.5), exact
  float a, b;      // slopes of the ray u = (a, b, 1)
  float uu;        // |u|^2
  float inv_uu;    // 1 / |u|^2 (hardware reciprocal)
};

__device__ __forceinline__ float rcp_approx(float x);

__device__ __forceinline__ PixRay pix_ray(const ViewParams &v, int px, int py) {
  PixRay r;
  r.pxc = (float)px + 0.5f;
  r.pyc = (float)py + 0.5f;
  r.a = __fmul_rn(__fsub_rn(r.pxc, v.cx), v.inv_f);
  r.b = __fmul_rn(__fsub_rn(v.cy, r.pyc), v.inv_f);
  r.uu = fmaf(r.a, r.a, fmaf(r.b, r.b, 1.0f));
  r.inv_uu = rcp_approx(r.uu);
  return r;
}

// sqrt(x) for x >= 0 by the hardware approximation (relative error near 2^-23; 0 gives 0).
__device__ __forceinline__ float sqrt_approx(float x) {
  float r;
  asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}

// ---------------------------------------------------------- precise setup --

struct Setup {
  df u0, v0;   // projection of the reference point (pixels)
  float zr;    // reference depth (FP32)
  float dz;    // zr - centre depth (0 unless the primitive reaches the eye plane)
  float k;     // zr / f: Angstrom per pixel at the reference depth
  float zc;    // centre depth (FP32)
  long long keyc;
};

// 64-bit integer <-> float conversions run on the FP64 pipe, which GB300 has
// at a small fraction of its FP32 rate; every conversion below therefore
// takes a 32-bit one when the value fits (the same result) and leaves the
// 64-bit one to a separate, rarely called function, so that the common path
// never issues it (a ternary would let the compiler evaluate both sides).
static __device__ __noinline__ long long float_to_ll_wide(float x) { return llrintf(fminf(fmaxf(x, -4.0e18f), 4.0e18f)); }
static __device__ __noinline__ float ll_to_float_wide(long long d) { return (float)d; }

// rint(x) for an integer-valued x (a float that already holds an integer)
__device__ __forceinline__ long long float_to_ll(float x) {
  if (x >= 0.0f && x < 4294967296.0f) return (long long)__float2uint_rn(x);
  if (x < 0.0f && x > -2147483648.0f) return (long long)__float2int_rn(x);
  return float_to_ll_wide(x);
}

// rint(x) as a 64-bit integer for any x (the 32-bit conversion when it fits)
__device__ __forceinline__ long long round_ll(float x) {
  if (fabsf(x) < 2.0e9f) return (long long)__float2int_rn(x);
  return float_to_ll_wide(x);
}

__device__ __forceinline__ long long key_of(df z, float zlo, float S) {
  df m = df_mul_f(df_add_f(z, -zlo), S);
  float h = rintf(m.hi);
  float fr = __fadd_rn(__fsub_rn(m.hi, h), m.lo);
  return float_to_ll(h) + (long long)__float2int_rn(fr);
}

// d = X - eye as double-floats (exact for float32 inputs).
// Rb: bounding radius (the reference depth is pushed to Rb + znear for a
// primitive that reaches the eye plane, so the projection stays finite).
__device__ __forceinline__ Setup precise_setup(const ViewParams &v, df dx, df dy, df dzw, float Rb, float zlo,
                                               float S) {
  df vx = df_dot3_lean(v.R, dx, dy, dzw);
  df vy = df_dot3_lean(v.U, dx, dy, dzw);
  df z = df_dot3_lean(v.F, dx, dy, dzw);
  Setup o;
  float zmin = Rb + v.znear;
  df zr = z;
  o.dz = 0.0f;
  if (z.hi < zmin) {
    zr = df{zmin, 0.0f};
    df dd = df_add(zr, df_neg(z));
    o.dz = dd.hi + dd.lo;
  }
  df fdf{v.f_hi, v.f_lo};
  df qx = df_div_lean(vx, zr), qy = df_div_lean(vy, zr);
  o.u0 = df_add_f(df_mul_lean(qx, fdf), v.cx);
  o.v0 = df_add_f(df_neg(df_mul_lean(qy, fdf)), v.cy);
  o.zr = zr.hi;
  o.zc = z.hi + z.lo;
  o.k = zr.hi * v.inv_f;
  o.keyc = key_of(zr, zlo, S);
  return o;
}

__device__ __forceinline__ void eye_offset(const ViewParams &v, float4 X, df &dx, df &dy, df &dz) {
  dx = two_sum(X.x, -v.eye[0]);
  dy = two_sum(X.y, -v.eye[1]);
  dz = two_sum(X.z, -v.eye[2]);
}

// Vector from the primitive's reference point to the pixel ray's point at
// the reference depth (internal frame).  Every component is Angstrom-scale.
__device__ __forceinline__ float3 local_o(float u0h, float u0l, float v0h, float v0l, float k, float dz,
                                          const PixRay &r) {
  float ox = __fsub_rn(__fsub_rn(r.pxc, u0h), u0l);
  float oy = __fsub_rn(__fsub_rn(r.pyc, v0h), v0l);
  return make_float3(__fmul_rn(k, ox), __fmul_rn(-k, oy), dz);
}

// Entry parameter s (depth = zr + s) of the ray o + s u into a sphere of radius rad at the origin.
// The hit tests spell every product-sum as an explicit fmaf or a plain
// operation, leaving the compiler no contraction choice: the direct-splat and
// binned paths, inlined into different kernels, then produce the same key bits.
// The square root and the division by |u|^2 use the hardware approximations
// (s is Angstrom-scale, so their ~1e-7 relative error is far below a depth-key
// step or the 1e-4 A tie band).
__device__ __forceinline__ bool sphere_local(float3 o, const PixRay &r, float rad, float &s) {
  float ou = fmaf(o.x, r.a, fmaf(o.y, r.b, o.z));
  float oo = fmaf(o.x, o.x, fmaf(o.y, o.y, __fmul_rn(o.z, o.z)));
  float disc = fmaf(ou, ou, __fmul_rn(-r.uu, fmaf(-rad, rad, oo)));
  if (!(disc >= 0.0f)) return false;
  s = __fmul_rn(__fsub_rn(-ou, sqrt_approx(disc)), r.inv_uu);
  return true;
}
__device__ __forceinline__ bool cylinder_local(float3 o, const PixRay &r, float3 A, float hl, float rb, float &s,
                                               int &kind, float &axial) {
  float ua = fmaf(r.a, A.x, fmaf(r.b, A.y, A.z));
  float oa = fmaf(o.x, A.x, fmaf(o.y, A.y, __fmul_rn(o.z, A.z)));
  float3 up = make_float3(fmaf(-ua, A.x, r.a), fmaf(-ua, A.y, r.b), fmaf(-ua, A.z, 1.0f));
  float3 op = make_float3(fmaf(-oa, A.x, o.x), fmaf(-oa, A.y, o.y), fmaf(-oa, A.z, o.z));
  float a2 = fmaf(up.x, up.x, fmaf(up.y, up.y, __fmul_rn(up.z, up.z)));
  float b2 = fmaf(op.x, up.x, fmaf(op.y, up.y, __fmul_rn(op.z, up.z)));
  float c2 = fmaf(-rb, rb, fmaf(op.x, op.x, fmaf(op.y, op.y, __fmul_rn(op.z, op.z))));
  const float rb2 = __fmul_rn(rb, rb);
  float best = __int_as_float(0x7f800000);
  kind = 0;
  if (a2 > 1e-12f) {
    float disc = fmaf(b2, b2, __fmul_rn(-a2, c2));
    if (disc >= 0.0f) {
      float s1 = __fdiv_rn(__fsub_rn(-b2, sqrtf(disc)), a2);
      float ax = fmaf(s1, ua, oa);
      if (fabsf(ax) <= hl) {
        best = s1;
        kind = 1;
      }
    }
  }
  if (fabsf(ua) > 1e-12f) {
#pragma unroll
    for (int sg = 0; sg < 2; ++sg) {
      float tgt = sg == 0 ? hl : -hl;
      float sc = __fdiv_rn(__fsub_rn(tgt, oa), ua);
      float qx = fmaf(sc, up.x, op.x), qy = fmaf(sc, up.y, op.y), qz = fmaf(sc, up.z, op.z);
      float rad2 = fmaf(qx, qx, fmaf(qy, qy, __fmul_rn(qz, qz)));
      if (rad2 <= rb2 && sc < best) {
        best = sc;
        kind = sg == 0 ? 2 : 3;
      }
    }
  }
  if (kind == 0) return false;
  s = best;
  axial = fmaf(s, ua, oa);
  return true;
}

// The offset s S is rounded to the nearest integer, through the 32-bit conversion whenever it fits
// (the same result as the 64-bit one, which is kept for the extreme key scales near the eye).
__device__ __forceinline__ unsigned long long pack_key(long long keyc, float s, float S, uint32_t id) {
  const float x = s * S;
  long long d;
  if (fabsf(x) < 2.0e9f)
    d = (long long)__float2int_rn(x);
  else
    d = float_to_ll_wide(x);
  long long k = keyc + d;
  k = k < 0 ? 0 : (k > kKeySpan ? kKeySpan : k);
  return ((unsigned long long)k << 32) | (unsigned long long)id;
}

// --------------------------------------------------- conservative bounds --

struct PixBox {
  int x0, x1, y0, y1;  // inclusive pixel-index ranges; empty when x0 > x1 or y0 > y1
};

// Pixel centres that a sphere (FP32 view centre vx, vy, depth z; radius R,
// centre error bound errR) can cover.  Exact per-axis tangent-slope bounds
// of the perspective projection, widened by an FP32 error margin.  Returns
// false when the sphere cannot produce an accepted hit.
__device__ __forceinline__ bool sphere_box(const ViewParams &v, int W, int H, float vx, float vy, float z, float R,
                                           float errR, PixBox &b) {
  float Rm = R + errR;
  if (z + Rm < v.znear) return false;
  if (z <= Rm * 1.01f) {  // reaches the eye plane: any pixel
    b.x0 = 0;
    b.x1 = W - 1;
    b.y0 = 0;
    b.y1 = H - 1;
    return true;
  }
  float zm = z - Rm, zp = z + Rm;
  float den = zm * zp;
  float sx = sqrtf(fmaf(vx, vx, den)), sy = sqrtf(fmaf(vy, vy, den));
  float mx0 = (vx * z - Rm * sx) / den, mx1 = (vx * z + Rm * sx) / den;
  float my0 = (vy * z - Rm * sy) / den, my1 = (vy * z + Rm * sy) / den;
  float mmax = fmaxf(fmaxf(fabsf(mx0), fabsf(mx1)), fmaxf(fabsf(my0), fabsf(my1)));
  float mpx = 1e-4f + v.f * (mmax + 1.0f) * (1e-6f + 4e-7f * z / zm);
  float X0 = v.cx + v.f * mx0 - mpx, X1 = v.cx + v.f * mx1 + mpx;
  float Y0 = v.cy - v.f * my1 - mpx, Y1 = v.cy - v.f * my0 + mpx;
  X0 = fmaxf(X0, -2.0f);
  Y0 = fmaxf(Y0, -2.0f);
  X1 = fminf(X1, (float)W + 2.0f);
  Y1 = fminf(Y1, (float)H + 2.0f);
  b.x0 = max((int)ceilf(X0 - 0.5f), 0);
  b.x1 = min((int)floorf(X1 - 0.5f), W - 1);
  b.y0 = max((int)ceilf(Y0 - 0.5f), 0);
  b.y1 = min((int)floorf(Y1 - 0.5f), H - 1);
  return b.x0 <= b.x1 && b.y0 <= b.y1;
}

// Cheap conservative streaming test: can the sphere (FP32 view centre, radius
// R, centre error err) cover a pixel centre with an entry point at or beyond
// the near plane?  One correctly rounded reciprocal and no division or square
// root.  The exact x-extent of a projected sphere around the projected
// centre m = vx/z is bounded by rho (|m| rho + sqrt(1 + m^2)) / (1 - rho^2),
// rho = R/z (tangent lines in the x-z plane; same for y), which is relaxed
// here to rho (1 + 2 rho^2)(|m| rho + 1 + m^2/2) for rho <= 1/8.  Larger or
// nearer spheres always survive (the precise setup decides).  The box then
// contains a pixel centre iff the nearest on-screen centre column and row do.
__device__ __forceinline__ bool cull_fast(const ViewParams &v, int W, int H, float vx, float vy, float z, float R,
                                          float err) {
  const float Rm = R + err;
  if (z + Rm < v.znear) return false;
  if (!(z > 8.0f * Rm)) return true;
  const float rz = __frcp_rn(z);
  const float rho = Rm * rz;
  const float mx = vx * rz, my = vy * rz;
  const float k = rho * fmaf(2.0f * rho, rho, 1.0f);
  const float hx = v.f * k * fmaf(fabsf(mx), rho, fmaf(0.5f * mx, mx, 1.0f));
  const float hy = v.f * k * fmaf(fabsf(my), rho, fmaf(0.5f * my, my, 1.0f));
  const float ux = fmaf(v.f, mx, v.cx - 0.5f), uy = fmaf(-v.f, my, v.cy - 0.5f);
  // FP32 rounding of this test (reciprocal, products, the pixel coordinate itself)
  const float ex = 1e-4f + 4e-6f * hx + 4e-7f * v.f * (fabsf(mx) + 1.0f) + 2.5e-7f * fabsf(ux);
  const float ey = 1e-4f + 4e-6f * hy + 4e-7f * v.f * (fabsf(my) + 1.0f) + 2.5e-7f * fabsf(uy);
  const float nx = fminf(fmaxf(rintf(ux), 0.0f), (float)(W - 1));
  const float ny = fminf(fmaxf(rintf(uy), 0.0f), (float)(H - 1));
  return fabsf(ux - nx) <= hx + ex && fabsf(uy - ny) <= hy + ey;
}

__device__ __forceinline__ float rcp_approx(float x) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}

// 2^x by the hardware approximation (relative error near 2^-22, flushes subnormals).
__device__ __forceinline__ float exp2_approx(float x) {
  float r;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}

// The same test as cull_fast with its rounding margins folded into per-view
// constants (ViewParams::hc, e0) and a 1-ulp approximate reciprocal:
//   reciprocal and products: <= 3.6e-7 relative on the slopes, i.e. at most
//   3.6e-7 (|u| + cx) px on the centre column u, and |u| <= W + h wherever
//   the test can pass; FP32 rounding of f: 6e-8 relative; rounding of h:
//   <= 7e-7 relative.  e0 = 1e-4 + 1e-6 (W + H) px and hc = f (1 + 4e-6)
//   cover these.  Rm already includes the error of the FP32 view centre.
__device__ __forceinline__ bool cull_lean(const ViewParams &v, float vx, float vy, float vz, float Rm) {
  if (!(vz + Rm >= v.znear)) return false;
  if (!(vz > 8.0f * Rm)) return true;
  const float rz = rcp_approx(vz);
  const float rho = Rm * rz;
  const float mx = vx * rz, my = vy * rz;
  const float t = v.hc * rho * fmaf(2.0f * rho, rho, 1.0f);
  const float hx = fmaf(t, fmaf(fabsf(mx), rho, fmaf(0.5f * mx, mx, 1.0f)), v.e0);
  const float hy = fmaf(t, fmaf(fabsf(my), rho, fmaf(0.5f * my, my, 1.0f)), v.e0);
  const float ux = fmaf(v.f, mx, v.cxm), uy = fmaf(-v.f, my, v.cym);
  const float nx = fminf(fmaxf(rintf(ux), 0.0f), v.wm1);
  const float ny = fminf(fmaxf(rintf(uy), 0.0f), v.hm1);
  return fabsf(ux - nx) <= hx && fabsf(uy - ny) <= hy;
}

// cull_lean and view_f32 for two atoms at once on the paired FP32 pipes
// (sm_100+ FFMA2/FMUL2/FADD2).  Each lane performs exactly the scalar
// operations of view_f32 / cull_lean in the same order, so the decisions are
// bit-identical to the scalar forms.
__device__ __forceinline__ float2 bc2(float a) { return make_float2(a, a); }

__device__ __forceinline__ void view_f32x2(const ViewParams &v, float2 x, float2 y, float2 z, float2 &vx, float2 &vy,
                                           float2 &vz, float2 &err) {
  const float2 dx = __fadd2_rn(x, bc2(-v.eye[0])), dy = __fadd2_rn(y, bc2(-v.eye[1])),
               dz = __fadd2_rn(z, bc2(-v.eye[2]));
  vx = __ffma2_rn(bc2(v.R[0]), dx, __ffma2_rn(bc2(v.R[1]), dy, __fmul2_rn(bc2(v.R[2]), dz)));
  vy = __ffma2_rn(bc2(v.U[0]), dx, __ffma2_rn(bc2(v.U[1]), dy, __fmul2_rn(bc2(v.U[2]), dz)));
  vz = __ffma2_rn(bc2(v.F[0]), dx, __ffma2_rn(bc2(v.F[1]), dy, __fmul2_rn(bc2(v.F[2]), dz)));
  err = make_float2(4e-7f * (fabsf(dx.x) + fabsf(dy.x) + fabsf(dz.x)), 4e-7f * (fabsf(dx.y) + fabsf(dy.y) + fabsf(dz.y)));
}

__device__ __forceinline__ void cull_lean_x2(const ViewParams &v, float2 vx, float2 vy, float2 vz, float2 Rm, bool &k0,
                                             bool &k1) {
  const float2 front = __fadd2_rn(vz, Rm);
  const float2 r8 = __fmul2_rn(bc2(8.0f), Rm);
  const float2 rz = make_float2(rcp_approx(vz.x), rcp_approx(vz.y));
  const float2 rho = __fmul2_rn(Rm, rz);
  const float2 mx = __fmul2_rn(vx, rz), my = __fmul2_rn(vy, rz);
  const float2 t = __fmul2_rn(__fmul2_rn(bc2(v.hc), rho), __ffma2_rn(__fmul2_rn(bc2(2.0f), rho), rho, bc2(1.0f)));
  const float2 amx = make_float2(fabsf(mx.x), fabsf(mx.y)), amy = make_float2(fabsf(my.x), fabsf(my.y));
  const float2 hx = __ffma2_rn(t, __ffma2_rn(amx, rho, __ffma2_rn(__fmul2_rn(bc2(0.5f), mx), mx, bc2(1.0f))), bc2(v.e0));
  const float2 hy = __ffma2_rn(t, __ffma2_rn(amy, rho, __ffma2_rn(__fmul2_rn(bc2(0.5f), my), my, bc2(1.0f))), bc2(v.e0));
  const float2 ux = __ffma2_rn(bc2(v.f), mx, bc2(v.cxm)), uy = __ffma2_rn(bc2(-v.f), my, bc2(v.cym));
  const float2 nx = make_float2(fminf(fmaxf(rintf(ux.x), 0.0f), v.wm1), fminf(fmaxf(rintf(ux.y), 0.0f), v.wm1));
  const float2 ny = make_float2(fminf(fmaxf(rintf(uy.x), 0.0f), v.hm1), fminf(fmaxf(rintf(uy.y), 0.0f), v.hm1));
  const float2 ex = __fadd2_rn(ux, make_float2(-nx.x, -nx.y)), ey = __fadd2_rn(uy, make_float2(-ny.x, -ny.y));
  k0 = front.x >= v.znear && (!(vz.x > r8.x) || (fabsf(ex.x) <= hx.x && fabsf(ey.x) <= hy.x));
  k1 = front.y >= v.znear && (!(vz.y > r8.y) || (fabsf(ex.y) <= hx.y && fabsf(ey.y) <= hy.y));
}

// Candidate pixel box of a sphere from the cull_lean bound (the exact
// tangent-slope box for spheres that come within 8 radii of the eye plane).
__device__ __forceinline__ bool lean_box(const ViewParams &v, int W, int H, float vx, float vy, float vz, float Rm,
                                         PixBox &b) {
  if (!(vz + Rm >= v.znear)) return false;
  if (!(vz > 8.0f * Rm)) return sphere_box(v, W, H, vx, vy, vz, Rm, 0.0f, b);
  const float rz = rcp_approx(vz);
  const float rho = Rm * rz;
  const float mx = vx * rz, my = vy * rz;
  const float t = v.hc * rho * fmaf(2.0f * rho, rho, 1.0f);
  const float hx = fmaf(t, fmaf(fabsf(mx), rho, fmaf(0.5f * mx, mx, 1.0f)), v.e0);
  const float hy = fmaf(t, fmaf(fabsf(my), rho, fmaf(0.5f * my, my, 1.0f)), v.e0);
  const float ux = fmaf(v.f, mx, v.cxm), uy = fmaf(-v.f, my, v.cym);
  b.x0 = (int)fminf(fmaxf(ceilf(ux - hx), 0.0f), (float)W);
  b.x1 = (int)fmaxf(fminf(floorf(ux + hx), (float)(W - 1)), -1.0f);
  b.y0 = (int)fminf(fmaxf(ceilf(uy - hy), 0.0f), (float)H);
  b.y1 = (int)fmaxf(fminf(floorf(uy + hy), (float)(H - 1)), -1.0f);
  return b.x0 <= b.x1 && b.y0 <= b.y1;
}

// ------------------------------------------------- TMA bulk copy helpers --
// Programmatic dependent launch (sm_90+ PTX): wait until the preceding grid
// of the stream has completed and its memory writes are visible (a no-op for
// a kernel launched without programmatic serialisation), then allow the next
// grid to begin launching.  Called first thing in every frame kernel.
__device__ __forceinline__ void pdl_enter() {
  asm volatile("griddepcontrol.wait;" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// 1-D bulk copies global -> shared completed on an mbarrier (sm_90+ PTX).

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }

__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}

__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_u32(dst)),
               "l"(src), "r"(bytes), "r"(smem_u32(bar))
               : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0u;
}

// Bounded wait: gives up after `limit` polls (each poll may suspend briefly).
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity, uint32_t limit) {
  for (uint32_t i = 0; i < limit; ++i)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}

// 16-byte asynchronous copies global -> shared (sm_80+ PTX), completed per thread in commit groups; the
// L2-only variant (.cg) leaves L1 to the kernel's other loads.
__device__ __forceinline__ void cp_async16(void *dst_smem, const void *src_gmem) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(dst_smem)), "l"(src_gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
// Wait until at most N of the calling thread's commit groups are still in flight.
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// Plain (non-transaction) arrival of the calling thread.
__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// FP32 view coordinates of a world point and the bound on their error.
__device__ __forceinline__ void view_f32(const ViewParams &v, float x, float y, float z, float &vx, float &vy,
                                         float &vz, float &err) {
  float dx = x - v.eye[0], dy = y - v.eye[1], dz = z - v.eye[2];
  vx = fmaf(v.R[0], dx, fmaf(v.R[1], dy, v.R[2] * dz));
  vy = fmaf(v.U[0], dx, fmaf(v.U[1], dy, v.U[2] * dz));
  vz = fmaf(v.F[0], dx, fmaf(v.F[1], dy, v.F[2] * dz));
  err = 4e-7f * (fabsf(dx) + fabsf(dy) + fabsf(dz));
}

// ------------------------------------------------------------- shading --

__device__ __forceinline__ float3 blinn_phong(const ShadeParams &sh, float3 n, const PixRay &r, float3 alb) {
  if (sh.model == 1) return alb;
  if (sh.model == 2 || sh.model == 3) {
    const float nl = fmaxf(n.x * sh.L[0] + n.y * sh.L[1] + n.z * sh.L[2], 0.0f);
    float b = nl;
    if (sh.model == 3) {
      const float lv = (float)sh.toon_levels;
      b = fminf(floorf(nl * lv), lv - 1.0f) / (lv - 1.0f);
    }
    const float d = sh.ka + sh.kd * b;
    return make_float3(fminf(alb.x * d, 1.0f), fminf(alb.y * d, 1.0f), fminf(alb.z * d, 1.0f));
  }
  float inv = 1.0f / sqrtf(r.uu);
  float3 V = make_float3(-r.a * inv, -r.b * inv, inv);
  float3 Hv = make_float3(sh.L[0] + V.x, sh.L[1] + V.y, sh.L[2] + V.z);
  float hinv = 1.0f / sqrtf(Hv.x * Hv.x + Hv.y * Hv.y + Hv.z * Hv.z);
  float nl = n.x * sh.L[0] + n.y * sh.L[1] + n.z * sh.L[2];
  float nh = (n.x * Hv.x + n.y * Hv.y + n.z * Hv.z) * hinv;
  float diff = sh.ka + sh.kd * fmaxf(nl, 0.0f);
  float spec = nl > 0.0f ? sh.ks * powf(fmaxf(nh, 0.0f), sh.shin) : 0.0f;
  return make_float3(fminf(fmaxf(alb.x * diff + spec, 0.0f), 1.0f), fminf(fmaxf(alb.y * diff + spec, 0.0f), 1.0f),
                     fminf(fmaxf(alb.z * diff + spec, 0.0f), 1.0f));
}

}  // namespace vtx
