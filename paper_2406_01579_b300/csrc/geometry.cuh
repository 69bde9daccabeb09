// Per-(view, tet) geometry shared by the preprocess kernel (which writes the
// blend record) and the record->vertex backward kernel (which recomputes the
// same intermediates and applies their adjoint).
#pragma once

#include "tets_internal.cuh"

namespace tts {

struct TetIn {
  float3 v[4];   // world-space vertices
  float f[4];    // vertex SDF
  float3 c[4];   // vertex colours
};

struct Geo {
  bool visible;
  unsigned int zbits;      // FP32 mean camera depth (sort key)
  float zbar;
  int i0, i1, j0, j1;      // pixel bbox (inclusive)
  // Pixel-scaled camera frame: xi = (fx x_c, fy y_c, z_c).  In it the ray of
  // pixel (px, py) has the exact direction (px - cx, py - cy, 1).
  float3 xm;               // centroid (high part of a double-float)
  float3 y[4];             // vertex offsets from the centroid (from world differences)
  float zr;                // reference depth
  float3 dr;               // reference ray direction (u_r - cx, v_r - cy, 1), exact
  float3 w;                // x_r - centroid, x_r = zr * dr (accurate: double-float centroid)
  float3 n[4];             // outward face normals (face k opposite vertex k)
  float e[4];              // plane offsets n . x_i (clamped away from 0)
  float sgn[4];            // orientation sign applied to (y_j - y_i) x (y_l - y_i)
  int slot_of[4];          // record slot of face k (front faces first, in face order)
  int nf;                  // number of front faces
  float3 g;                // SDF gradient in the pixel-scaled frame
  float3 cof[3];           // cofactor columns of the edge matrix
  float det;               // 6 * signed volume (pixel-scaled frame)
  float fm, fr;            // SDF at the centroid and at x_r
  float P[4], A[4], B[4];  // per slot
};

__device__ __forceinline__ float3 f3(float x, float y, float z) { return make_float3(x, y, z); }
__device__ __forceinline__ float3 operator+(float3 a, float3 b) { return f3(a.x + b.x, a.y + b.y, a.z + b.z); }
__device__ __forceinline__ float3 operator-(float3 a, float3 b) { return f3(a.x - b.x, a.y - b.y, a.z - b.z); }
__device__ __forceinline__ float3 operator*(float s, float3 a) { return f3(s * a.x, s * a.y, s * a.z); }
__device__ __forceinline__ float dot3(float3 a, float3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
__device__ __forceinline__ float3 cross3(float3 a, float3 b) {
  return f3(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}
__device__ __forceinline__ float3 rot(const float* R, float3 v) {
  return f3(R[0] * v.x + R[1] * v.y + R[2] * v.z, R[3] * v.x + R[4] * v.y + R[5] * v.z,
            R[6] * v.x + R[7] * v.y + R[8] * v.z);
}
__device__ __forceinline__ float3 rotT(const float* R, float3 v) {
  return f3(R[0] * v.x + R[3] * v.y + R[6] * v.z, R[1] * v.x + R[4] * v.y + R[7] * v.z,
            R[2] * v.x + R[5] * v.y + R[8] * v.z);
}

// Error-free transformations (Knuth TwoSum, FMA-based TwoProduct) for the
// double-float centroid transform; explicit roundings keep them exact.
struct DF {
  float hi, lo;
};
__device__ __forceinline__ DF two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float z = __fsub_rn(s, a);
  const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, z)), __fsub_rn(b, z));
  return {s, e};
}
__device__ __forceinline__ DF two_prod(float a, float b) {
  const float p = __fmul_rn(a, b);
  return {p, __fmaf_rn(a, b, -p)};
}
__device__ __forceinline__ DF df_norm(DF x) {
  const float s = __fadd_rn(x.hi, x.lo);
  return {s, __fsub_rn(x.lo, __fsub_rn(s, x.hi))};
}
// scale * (r0 a + r1 b + r2 c + t) with ~48-bit accuracy
__device__ __forceinline__ DF df_affine(float r0, float r1, float r2, float t, float a, float b,
                                        float c, float scale) {
  DF acc = two_prod(r0, a);
  DF p = two_prod(r1, b);
  DF s = two_sum(acc.hi, p.hi);
  acc = {s.hi, __fadd_rn(__fadd_rn(acc.lo, p.lo), s.lo)};
  p = two_prod(r2, c);
  s = two_sum(acc.hi, p.hi);
  acc = {s.hi, __fadd_rn(__fadd_rn(acc.lo, p.lo), s.lo)};
  s = two_sum(acc.hi, t);
  acc = df_norm({s.hi, __fadd_rn(acc.lo, s.lo)});
  p = two_prod(scale, acc.hi);
  return df_norm({p.hi, __fmaf_rn(scale, acc.lo, p.lo)});
}

__constant__ static const int kFaceVerts[4][3] = {{1, 2, 3}, {0, 2, 3}, {0, 1, 3}, {0, 1, 2}};

// The binning key path: an exact FP32 op sequence (the CPU checker replays
// it bit for bit).  Returns false when the tet is culled (near plane or an
// empty pixel bbox).
__device__ __forceinline__ bool key_path(const ViewD& vw, const TetIn& in, Geo& G,
                                         float* pu = nullptr, float* pv = nullptr) {
  float x[4], y[4], z[4];
  bool cull = false;
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const float3 v = in.v[j];
    x[j] = __fmaf_rn(vw.R[0], v.x, __fmaf_rn(vw.R[1], v.y, __fmaf_rn(vw.R[2], v.z, vw.t[0])));
    y[j] = __fmaf_rn(vw.R[3], v.x, __fmaf_rn(vw.R[4], v.y, __fmaf_rn(vw.R[5], v.z, vw.t[1])));
    z[j] = __fmaf_rn(vw.R[6], v.x, __fmaf_rn(vw.R[7], v.y, __fmaf_rn(vw.R[8], v.z, vw.t[2])));
    cull |= !(z[j] >= vw.znear);
  }
  G.zbar = __fmul_rn(__fadd_rn(__fadd_rn(z[0], z[1]), __fadd_rn(z[2], z[3])), 0.25f);
  G.zbits = __float_as_uint(G.zbar);
  if (cull) return false;
  float umin = INFINITY, umax = -INFINITY, vmin = INFINITY, vmax = -INFINITY;
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const float u = __fmaf_rn(vw.fx, __fdiv_rn(x[j], z[j]), vw.cx);
    const float v = __fmaf_rn(vw.fy, __fdiv_rn(y[j], z[j]), vw.cy);
    if (pu) pu[j] = u;
    if (pv) pv[j] = v;
    umin = fminf(umin, u); umax = fmaxf(umax, u);
    vmin = fminf(vmin, v); vmax = fmaxf(vmax, v);
  }
  const float i0 = fmaxf(ceilf(__fsub_rn(umin, 0.5f)), 0.f);
  const float i1 = fminf(floorf(__fsub_rn(umax, 0.5f)), (float)(vw.W - 1));
  const float j0 = fmaxf(ceilf(__fsub_rn(vmin, 0.5f)), 0.f);
  const float j1 = fminf(floorf(__fsub_rn(vmax, 0.5f)), (float)(vw.H - 1));
  if (!(i0 <= i1) || !(j0 <= j1)) return false;
  G.i0 = (int)i0; G.i1 = (int)i1; G.j0 = (int)j0; G.j1 = (int)j1;
  return true;
}

// Hull test of the tile rect (TTS_FLAG_HULL): the tet's projection is the
// convex hull of its four projected vertices; a tile of the rect is kept
// unless, for some hull edge, all four corner pixel centres of (tile x pixel
// bbox) lie strictly outside it.  An exact FP32 op sequence (the CPU checker
// replays it bit for bit): for the edge (a, b) and a point p,
//   E = fma(bu - au, pv - av, -((bv - av) * (pu - au)))
// and (a, b) is a hull edge when E has the same nonzero sign at the other two
// vertices.  Rects of two to HULL_MAX x HULL_MAX tiles are tested (one-tile
// rects and wider or taller ones keep every tile); the kept cells come back
// as a mask, bit cy * ntx + cx.  Per hull edge the factors (pv - av) of each row's two
// corner heights and (bv - av) * (pu - au) of each column's two corner
// abscissae are formed once and each corner costs one fma.
constexpr int HULL_MAX = 2;

__device__ __forceinline__ unsigned hull_tile_mask(const float pu[4], const float pv[4], const Geo& G,
                                                   int tsh, int tx0, int ty0, int ntx, int nty) {
  const int nt = ntx * nty;
  const unsigned all = (nt >= 32) ? 0xffffffffu : ((1u << nt) - 1u);
  // one-tile rects are not tested (only a sliver whose hull holds no pixel
  // centre of its bbox could lose its key), nor rects of more than
  // HULL_MAX tiles in a direction
  if (nt == 1 || ntx > HULL_MAX || nty > HULL_MAX) return all;
  const int T = 1 << tsh;
  float xl[HULL_MAX], xr[HULL_MAX], yl[HULL_MAX], yr[HULL_MAX];
#pragma unroll
  for (int c = 0; c < HULL_MAX; ++c) {
    const int tx = (tx0 + c) << tsh, ty = (ty0 + c) << tsh;
    xl[c] = (float)max(tx, G.i0) + 0.5f;
    xr[c] = (float)min(tx + T - 1, G.i1) + 0.5f;
    yl[c] = (float)max(ty, G.j0) + 0.5f;
    yr[c] = (float)min(ty + T - 1, G.j1) + 0.5f;
  }
  unsigned keep = all;
  constexpr int PA[6] = {0, 0, 0, 1, 1, 2}, PB[6] = {1, 2, 3, 2, 3, 3};
  constexpr int PC[6] = {2, 1, 1, 0, 0, 0}, PD[6] = {3, 3, 2, 3, 2, 1};
#pragma unroll
  for (int e = 0; e < 6; ++e) {
    const float au = pu[PA[e]], av = pv[PA[e]];
    const float ex = __fsub_rn(pu[PB[e]], au), ey = __fsub_rn(pv[PB[e]], av);
    const float ec = __fmaf_rn(ex, __fsub_rn(pv[PC[e]], av), -__fmul_rn(ey, __fsub_rn(pu[PC[e]], au)));
    const float ed = __fmaf_rn(ex, __fsub_rn(pv[PD[e]], av), -__fmul_rn(ey, __fsub_rn(pu[PD[e]], au)));
    if (!((ec > 0.f && ed > 0.f) || (ec < 0.f && ed < 0.f))) continue;   // not a hull edge
    const float sg = (ec > 0.f) ? 1.f : -1.f;   // the hull's side of the edge
    float Al[HULL_MAX], Ar[HULL_MAX], Bl[HULL_MAX], Br[HULL_MAX];
#pragma unroll
    for (int c = 0; c < HULL_MAX; ++c) {
      Al[c] = __fmul_rn(ey, __fsub_rn(xl[c], au));
      Ar[c] = __fmul_rn(ey, __fsub_rn(xr[c], au));
      Bl[c] = __fsub_rn(yl[c], av);
      Br[c] = __fsub_rn(yr[c], av);
    }
#pragma unroll
    for (int r = 0; r < HULL_MAX; ++r) {
#pragma unroll
      for (int c = 0; c < HULL_MAX; ++c) {
        if (r < nty && c < ntx) {
          // strictly outside at all four corners: sg * E < 0 (sg * E is exact)
          const float m = fmaxf(fmaxf(sg * __fmaf_rn(ex, Bl[r], -Al[c]), sg * __fmaf_rn(ex, Bl[r], -Ar[c])),
                                fmaxf(sg * __fmaf_rn(ex, Br[r], -Al[c]), sg * __fmaf_rn(ex, Br[r], -Ar[c])));
          if (m < 0.f) keep &= ~(1u << (r * ntx + c));
        }
      }
    }
  }
  return keep;
}

// Full per-(view, tet) geometry, in the pixel-scaled camera frame.  The chord
// parametrisation is relative to the tet: vertex offsets come from world-space
// differences and the centroid's camera position is a double-float, so the
// offset between the tet and the reference pixel ray carries no rounding at
// the scale of the camera distance (which the Eq. 1 steepness s would
// amplify).
__device__ __forceinline__ void tet_geometry_rest(const ViewD& vw, const TetIn& in, Geo& G);

__device__ __forceinline__ void tet_geometry(const ViewD& vw, float s, const TetIn& in, Geo& G) {
  (void)s;
  G.visible = key_path(vw, in, G);
  if (!G.visible) return;
  tet_geometry_rest(vw, in, G);
}

// The same geometry for a tet whose key path already ran (in the forward): the
// pixel bbox corner (i0, j0) comes from its record instead.  zbits, zbar and
// (i1, j1) are not set.
__device__ __forceinline__ void tet_geometry_at(const ViewD& vw, const TetIn& in, int i0, int j0,
                                                Geo& G) {
  G.visible = true;
  G.i0 = i0;
  G.j0 = j0;
  tet_geometry_rest(vw, in, G);
}

// Everything after the key path: frame, reference point, faces, affine SDF.
__device__ __forceinline__ void tet_geometry_rest(const ViewD& vw, const TetIn& in, Geo& G) {
  const float sx = vw.fx, sy = vw.fy;
  const float3 m = 0.25f * ((in.v[0] + in.v[1]) + (in.v[2] + in.v[3]));
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const float3 c = rot(vw.R, in.v[j] - m);
    G.y[j] = f3(sx * c.x, sy * c.y, c.z);
  }
  const DF mx = df_affine(vw.R[0], vw.R[1], vw.R[2], vw.t[0], m.x, m.y, m.z, sx);
  const DF my = df_affine(vw.R[3], vw.R[4], vw.R[5], vw.t[1], m.x, m.y, m.z, sy);
  const DF mz = df_affine(vw.R[6], vw.R[7], vw.R[8], vw.t[2], m.x, m.y, m.z, 1.f);
  G.xm = f3(mx.hi, my.hi, mz.hi);
  // reference point: on the ray through the bbox corner pixel centre, at depth zr
  G.zr = mz.hi;
  G.dr = f3((float)G.i0 + 0.5f - vw.cx, (float)G.j0 + 0.5f - vw.cy, 1.f);
  G.w = f3(__fsub_rn(__fmaf_rn(G.zr, G.dr.x, -mx.hi), mx.lo),
           __fsub_rn(__fmaf_rn(G.zr, G.dr.y, -my.hi), my.lo), -mz.lo);
  // edge matrix (rows y_j - y_0) and its cofactors
  const float3 Y0 = G.y[1] - G.y[0], Y1 = G.y[2] - G.y[0], Y2 = G.y[3] - G.y[0];
  G.cof[0] = cross3(Y1, Y2);
  G.cof[1] = cross3(Y2, Y0);
  G.cof[2] = cross3(Y0, Y1);
  G.det = dot3(Y0, G.cof[0]);
  const float l2 = fmaxf(fmaxf(dot3(Y0, Y0), dot3(Y1, Y1)), dot3(Y2, Y2));
  if (!(fabsf(G.det) > 1e-9f * l2 * sqrtf(l2))) { G.visible = false; return; }   // flat tet
  int nf = 0;
  float Pf[4], Af[4], Bf[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const int i = kFaceVerts[k][0], j = kFaceVerts[k][1], l = kFaceVerts[k][2];
    float3 n = cross3(G.y[j] - G.y[i], G.y[l] - G.y[i]);
    float sg = 1.f;
    if (dot3(n, G.y[k] - G.y[i]) > 0.f) { n = -1.f * n; sg = -1.f; }
    float e = dot3(n, G.xm) + dot3(n, G.y[i]);
    const float emin = 1e-7f * (fabsf(n.x * G.xm.x) + fabsf(n.y * G.xm.y) + fabsf(n.z * G.xm.z));
    if (fabsf(e) < emin) e = (e < 0.f) ? -emin : emin;
    G.n[k] = n;
    G.e[k] = e;
    G.sgn[k] = sg;
    const float inv = rcp_approx(e);   // |e| is clamped away from 0 above
    Pf[k] = dot3(n, G.w - G.y[i]) * inv;
    Af[k] = G.zr * n.x * inv;
    Bf[k] = G.zr * n.y * inv;
    nf += (e < 0.f);
  }
  G.nf = nf;
  if (nf == 0 || nf == 4) { G.visible = false; return; }
  // slots: front faces first, then back faces, each in face order
  int fb = 0;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const bool front = G.e[k] < 0.f;
    G.slot_of[k] = front ? fb : nf + (k - fb);
    fb += front;
  }
#pragma unroll
  for (int sl = 0; sl < 4; ++sl) {
    G.P[sl] = (G.slot_of[0] == sl) ? Pf[0] : (G.slot_of[1] == sl) ? Pf[1] : (G.slot_of[2] == sl) ? Pf[2] : Pf[3];
    G.A[sl] = (G.slot_of[0] == sl) ? Af[0] : (G.slot_of[1] == sl) ? Af[1] : (G.slot_of[2] == sl) ? Af[2] : Af[3];
    G.B[sl] = (G.slot_of[0] == sl) ? Bf[0] : (G.slot_of[1] == sl) ? Bf[1] : (G.slot_of[2] == sl) ? Bf[2] : Bf[3];
  }
  // affine SDF: gradient g from the edge system, value at the reference point
  const float d1 = in.f[1] - in.f[0], d2 = in.f[2] - in.f[0], d3 = in.f[3] - in.f[0];
  const float idet = rcp_approx(G.det);   // a flat tet was rejected above
  G.g = idet * (d1 * G.cof[0] + d2 * G.cof[1] + d3 * G.cof[2]);
  G.fm = 0.25f * ((in.f[0] + in.f[1]) + (in.f[2] + in.f[3]));
  G.fr = G.fm + dot3(G.g, G.w);
}

// The tet's colour (R6): the mean of its vertex colours, in this sum order.
__device__ __forceinline__ float3 tet_colour(const float3 c[4]) {
  return 0.25f * ((c[0] + c[1]) + (c[2] + c[3]));
}

__device__ __forceinline__ void write_record(const ViewD& vw, float s, const TetIn& in, const Geo& G,
                                             float3 colour, float4* __restrict__ out) {
  (void)vw;
  const float bx = (float)G.i0 + 0.5f, by = (float)G.j0 + 0.5f;
  out[0] = make_float4((G.nf >= 2) ? -bx : bx, (G.nf >= 3) ? -by : by, (float)G.i1 + 0.5f,
                       (float)G.j1 + 0.5f);
  out[1] = make_float4(G.P[0], G.P[1], G.P[2], G.P[3]);
  out[2] = make_float4(G.A[0], G.A[1], G.A[2], G.A[3]);
  out[3] = make_float4(G.B[0], G.B[1], G.B[2], G.B[3]);
  const float sz = s * G.zr;
  const float F = s * G.fr;
  const float K0 = sz * dot3(G.g, G.dr);
  out[4] = make_float4(F, K0, sz * G.g.x, sz * G.g.y);
  out[5] = make_float4(G.zbar, colour.x, colour.y, colour.z);
}

// World-space SDF gradient of a tet (App. A.3).  With edge rows
// y_j = v_j - v_0 and d_j = f_j - f_0 (j = 1..3) the affine field has
// g = Y^-1 d = h / det, h = d_1 c_1 + d_2 c_2 + d_3 c_3, where c_1 = y_2 x y_3,
// c_2 = y_3 x y_1, c_3 = y_1 x y_2 are the cofactor columns and det = y_1 . c_1.
struct TetGrad {
  float3 y[3], c[3];
  float d[3];
  float3 h;      // det * g
  float det;
};

__device__ __forceinline__ void tet_grad(const float3 v[4], const float f[4], TetGrad& G) {
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    G.y[j] = v[j + 1] - v[0];
    G.d[j] = f[j + 1] - f[0];
  }
  G.c[0] = cross3(G.y[1], G.y[2]);
  G.c[1] = cross3(G.y[2], G.y[0]);
  G.c[2] = cross3(G.y[0], G.y[1]);
  G.h = G.d[0] * G.c[0] + G.d[1] * G.c[1] + G.d[2] * G.c[2];
  G.det = dot3(G.y[0], G.c[0]);
}

// Unit normal n = g / |g| = sign(det) h / |h| (Sec. 3.2 per-tet normal); zero
// for a flat tet or a constant field.  *inv_h = 1/|h| (0 when degenerate),
// *sg = sign(det).
__device__ __forceinline__ float3 tet_unit_normal(const TetGrad& G, float* inv_h, float* sg) {
  const float hh = dot3(G.h, G.h);
  *sg = (G.det < 0.f) ? -1.f : 1.f;
  if (!(hh > 0.f) || G.det == 0.f) {
    *inv_h = 0.f;
    return f3(0.f, 0.f, 0.f);
  }
  const float ih = 1.f / sqrtf(hh);
  *inv_h = ih;
  return (*sg * ih) * G.h;
}

// Adjoint of (h, det) -> (v, f): adds dL/dv_j and dL/df_j given dL/dh, dL/ddet.
__device__ __forceinline__ void tet_grad_adjoint(const TetGrad& G, float3 dh, float ddet,
                                                 float3 dv[4], float df[4]) {
  float3 dc[3], dy[3];
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    const float dd = dot3(G.c[j], dh);
    df[j + 1] += dd;
    df[0] -= dd;
    dc[j] = G.d[j] * dh;
  }
  // det = y_0 . c_0 with d det / d y_j = c_j
  dy[0] = cross3(dc[1], G.y[2]) + cross3(G.y[1], dc[2]) + ddet * G.c[0];
  dy[1] = cross3(G.y[2], dc[0]) + cross3(dc[2], G.y[0]) + ddet * G.c[1];
  dy[2] = cross3(dc[0], G.y[1]) + cross3(G.y[0], dc[1]) + ddet * G.c[2];
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    dv[j + 1] = dv[j + 1] + dy[j];
    dv[0] = dv[0] - dy[j];
  }
}

// Adjoint of the unit normal: dL/dh from dL/dn.
__device__ __forceinline__ float3 tet_normal_adjoint(float3 n, float inv_h, float sg, float3 dn) {
  return (sg * inv_h) * (dn - dot3(n, dn) * n);
}

// The vertices, SDF values and (when COLOURS) vertex colours of the tet with
// vertex ids t.
template <bool COLOURS = true>
__device__ __forceinline__ void load_tet_ids(const SceneD& S, int4 t, TetIn& in) {
  const int id[4] = {t.x, t.y, t.z, t.w};
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const float* v = S.V + 3ll * id[j];
    in.v[j] = f3(__ldg(v), __ldg(v + 1), __ldg(v + 2));
    in.f[j] = __ldg(S.f + id[j]);
    if constexpr (COLOURS) {
      const float* c = S.rgb + 3ll * id[j];
      in.c[j] = f3(__ldg(c), __ldg(c + 1), __ldg(c + 2));
    }
  }
}

}  // namespace tts
