// Oracle for the tetrahedron splatting rasterizer.  TEST INFRASTRUCTURE ONLY:
// only the test suite, the smoke check and the benchmark's CPU-baseline leg may
// load this library.  It shares no code with the CUDA path.
//
// A plain, slow CPU restatement of the method, in FP64 except for the binning
// key path, which is an exact FP32 op sequence (the GPU sorts FP32 keys and the
// key lists are compared bit for bit).
//
//   prefilter      Sec. 3.2 "Pre-filtering" + Eq. 1: alpha_max from the max and
//                  min vertex SDF, keep iff alpha_max >= T_f.
//   bin            Sec. 3.3: cull against the near plane and the image, pixel
//                  bbox -> tile rect, one key (tile, mean vertex depth) per
//                  overlapped tile, stable sort (ties: survivor order).
//   render         Sec. 3.2 + App. A.1/A.2: per pixel, every listed tet whose
//                  bbox holds the pixel is intersected through its four
//                  projected triangles (2D barycentrics, App. A.1), each hit is
//                  perspective corrected (App. A.2) to (z_p, f_p); the nearest
//                  and farthest hits give f_prev, f_next; Eq. 1 gives alpha;
//                  Eq. 2 composites front to back with the 3DGS conventions
//                  (cap 0.99, skip below 1/255, stop before T drops under 1e-4).
//   adjoint        exact derivatives: the compositing adjoint written out, and
//                  per-fragment d alpha / d(vertex xyz, vertex f) from
//                  forward-mode dual numbers through the same FP64 code.
//
// Parity status: pinned (closed forms, three-route chord agreement,
// telescoping identity, invariants, dual numbers, finite differences) except
// the decision-band alternative branch, which is a test aid.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <numeric>
#include <vector>
#ifdef _OPENMP
#include <omp.h>
#endif

extern "C" {

struct OrcCam {
  float R[9];
  float t[3];
  float fx, fy, cx, cy, znear;
  int32_t width, height;
};

struct OrcParams {
  double s;                 // Eq. 1 steepness
  double prefilter_thresh;  // T_f
  double alpha_skip;        // 3DGS skip threshold
  double alpha_cap;         // 3DGS cap
  double t_eps;             // 3DGS termination threshold
  double band;              // relative half-width of the decision bands
  int32_t tile;             // tile edge in pixels
  int32_t flags;            // bit 0: PURE (no cap, skip, termination, pre-filter)
  int32_t window;           // resort window N_w (Sec. 3.3); 0: tile order; <0: full per-pixel sort
  int32_t pad;
};

}  // extern "C"

static const int ORC_PURE = 1;

#include "dual.h"

// ---------------------------------------------------------------------------
// Eq. 1 in the exact rewrite that cannot form 0/0:
//   (Phi(fp) - Phi(fn)) / Phi(fp) = -expm1(-s (fp - fn)) * sigmoid(-s fn)
// and 0 when fp <= fn (the max(., 0) of Eq. 1).
// ---------------------------------------------------------------------------
template <class S>
static S opacity_eq1(const S& fp, const S& fn, double s) {
  if (!(val(fp) > val(fn))) return S(0.0);
  S a = -dexpm1(-(s * (fp - fn)));
  S b = 1.0 / (1.0 + dexp(s * fn));
  return a * b;
}

// ---------------------------------------------------------------------------
// one fragment: ray through pixel centre (px, py) against tet with camera-space
// vertices X[4][3] and vertex SDF F[4].  App. A.1 (2D barycentrics of the four
// projected triangles, closed inside test) and App. A.2 (perspective
// correction).  Returns false when the ray meets the tet in fewer than two
// distinct points.
// ---------------------------------------------------------------------------
template <class S>
struct FragOut {
  S f_prev, f_next, z_in, z_out;
  int k_in, k_out;    // faces giving the entry and the exit point
};

// One face of a tet against the ray of pixel centre (px, py): App. A.1's 2D
// barycentrics of the projected triangle (Cramer) and App. A.2's perspective
// correction of the depth z_p and the SDF f_p at the point where the ray meets
// the face's plane.  ok: the projected triangle is not edge-on; minb: the
// smallest of the three barycentrics (>= 0 inside the triangle).
template <class S>
struct FaceEval {
  bool ok;
  double minb;
  S z, f;
};

static const int kFaces[4][3] = {{1, 2, 3}, {0, 2, 3}, {0, 1, 3}, {0, 1, 2}};

template <class S>
static void eval_faces(const S X[4][3], const S F[4], double px, double py, double fx, double fy,
                       double cx, double cy, FaceEval<S> out[4]) {
  S u[4], v[4];
  for (int j = 0; j < 4; ++j) {
    u[j] = fx * (X[j][0] / X[j][2]) + cx;
    v[j] = fy * (X[j][1] / X[j][2]) + cy;
  }
  for (int k = 0; k < 4; ++k) {
    const int a = kFaces[k][0], b = kFaces[k][1], c = kFaces[k][2];
    out[k].ok = false;
    // [v_a' v_b' v_c'; 1 1 1] [1-u'-v', u', v']^T = [p; 1]  (App. A.1), Cramer
    S ub = u[b] - u[a], vb = v[b] - v[a], uc = u[c] - u[a], vc = v[c] - v[a];
    S det = ub * vc - uc * vb;
    double scale = std::fabs(val(ub) * val(vc)) + std::fabs(val(uc) * val(vb));
    if (!(std::fabs(val(det)) > 1e-14 * scale) || scale == 0.0) continue;  // edge-on face
    S qx = px - u[a], qy = py - v[a];
    S bu = (qx * vc - uc * qy) / det;   // u'
    S bv = (ub * qy - qx * vb) / det;   // v'
    S b0 = 1.0 - bu - bv;               // 1 - u' - v'
    // App. A.2: perspective-correct barycentrics and the interpolated SDF/depth
    S sig = b0 / X[a][2] + bu / X[b][2] + bv / X[c][2];
    S uu = (bu / X[b][2]) / sig;
    S vv = (bv / X[c][2]) / sig;
    out[k].f = (1.0 - uu - vv) * F[a] + uu * F[b] + vv * F[c];
    out[k].z = 1.0 / sig;
    out[k].minb = std::min(val(b0), std::min(val(bu), val(bv)));
    out[k].ok = true;
  }
}

// ---------------------------------------------------------------------------
// one fragment: ray through pixel centre (px, py) against tet with camera-space
// vertices X[4][3] and vertex SDF F[4].  The faces the ray hits (closed inside
// test); the nearest hit gives f_prev, the farthest f_next.  Returns false
// when the ray meets the tet in fewer than two distinct points.
// ---------------------------------------------------------------------------
template <class S>
static bool eval_fragment(const S X[4][3], const S F[4], double px, double py,
                          double fx, double fy, double cx, double cy,
                          FragOut<S>* out) {
  FaceEval<S> fe[4];
  eval_faces<S>(X, F, px, py, fx, fy, cx, cy, fe);
  const double tol = -1e-12;
  int imin = -1, imax = -1, nhit = 0;
  for (int k = 0; k < 4; ++k) {
    if (!fe[k].ok || fe[k].minb < tol) continue;
    ++nhit;
    if (imin < 0 || val(fe[k].z) < val(fe[imin].z)) imin = k;
    if (imax < 0 || val(fe[k].z) > val(fe[imax].z)) imax = k;
  }
  if (nhit < 2) return false;
  if (!(val(fe[imax].z) - val(fe[imin].z) > 1e-12 * val(fe[imax].z))) return false;
  out->f_prev = fe[imin].f;
  out->f_next = fe[imax].f;
  out->z_in = fe[imin].z;
  out->z_out = fe[imax].z;
  out->k_in = imin;
  out->k_out = imax;
  return true;
}

// Faces other than the chosen entry (exit) face whose plane the ray meets
// within rel_z of the entry (exit) depth, at a point within rel_b of their
// triangle: the ray passes that close to the edge they share with the chosen
// face, where the chord's entry (exit) point has a kink (its derivative with
// respect to the vertex positions depends on the face).  A computation in
// another precision may take either face.  Returns the candidates for the
// entry in alt_in[0..n_in) and for the exit in alt_out[0..n_out).
template <class S>
static void near_kink_faces(const S X[4][3], const S F[4], double px, double py, double fx,
                            double fy, double cx, double cy, const FragOut<S>& o, double rel_z,
                            double rel_b, int alt_in[4], int* n_in, int alt_out[4], int* n_out) {
  FaceEval<S> fe[4];
  eval_faces<S>(X, F, px, py, fx, fy, cx, cy, fe);
  *n_in = *n_out = 0;
  for (int k = 0; k < 4; ++k) {
    if (!fe[k].ok || fe[k].minb < -rel_b) continue;
    const double z = val(fe[k].z);
    if (k != o.k_in && std::fabs(z - val(o.z_in)) <= rel_z * val(o.z_in)) alt_in[(*n_in)++] = k;
    if (k != o.k_out && std::fabs(z - val(o.z_out)) <= rel_z * val(o.z_out)) alt_out[(*n_out)++] = k;
  }
}

// ---------------------------------------------------------------------------
// camera transform in FP64 (from the FP32 inputs)
// ---------------------------------------------------------------------------
static inline void cam_xform(const OrcCam& c, const double* v, double out[3]) {
  for (int r = 0; r < 3; ++r)
    out[r] = (double)c.R[3 * r] * v[0] + (double)c.R[3 * r + 1] * v[1] +
             (double)c.R[3 * r + 2] * v[2] + (double)c.t[r];
}

// FP64 view of the vertex data: the FP32 inputs widened, or caller-supplied
// FP64 overrides (finite-difference tests perturb those; the binning lists stay
// those of the FP32 inputs).
struct Fields {
  std::vector<double> V, f, rgb;
  Fields(int64_t N, const float* V32, const float* f32, const float* rgb32, const double* V64,
         const double* f64, const double* rgb64)
      : V(3 * N), f(N), rgb(3 * N) {
    for (int64_t i = 0; i < 3 * N; ++i) {
      V[i] = V64 ? V64[i] : (double)V32[i];
      rgb[i] = rgb64 ? rgb64[i] : (double)rgb32[i];
    }
    for (int64_t i = 0; i < N; ++i) f[i] = f64 ? f64[i] : (double)f32[i];
  }
};

// ---------------------------------------------------------------------------
// Per-tet normal (Sec. 3.2 "Per-tetrahedron normal", App. A.3): the SDF is
// affine in the tet, [g; c0] = [x_j^T 1]^{-1} f.  Solved here on the
// camera-space vertices by Gaussian elimination with partial pivoting, then
// taken to world space (g_w = R^T g, the chain rule of x = R v + t) and
// normalised.  Returns false for a zero gradient (normal 0).
// ---------------------------------------------------------------------------
template <class S>
static bool tet_normal_world(const S X[4][3], const S F[4], const OrcCam& c, S n[3]) {
  S M[4][5];
  for (int j = 0; j < 4; ++j) {
    for (int r = 0; r < 3; ++r) M[j][r] = X[j][r];
    M[j][3] = S(1.0);
    M[j][4] = F[j];
  }
  for (int col = 0; col < 4; ++col) {
    int piv = col;
    for (int r = col + 1; r < 4; ++r)
      if (std::fabs(val(M[r][col])) > std::fabs(val(M[piv][col]))) piv = r;
    if (val(M[piv][col]) == 0.0) return false;
    if (piv != col)
      for (int k = 0; k < 5; ++k) std::swap(M[piv][k], M[col][k]);
    for (int r = col + 1; r < 4; ++r) {
      const S fct = M[r][col] / M[col][col];
      for (int k = col; k < 5; ++k) M[r][k] = M[r][k] - fct * M[col][k];
    }
  }
  S sol[4];
  for (int r = 3; r >= 0; --r) {
    S acc = M[r][4];
    for (int k = r + 1; k < 4; ++k) acc = acc - M[r][k] * sol[k];
    sol[r] = acc / M[r][r];
  }
  S gw[3];
  for (int r = 0; r < 3; ++r)
    gw[r] = (double)c.R[r] * sol[0] + (double)c.R[3 + r] * sol[1] + (double)c.R[6 + r] * sol[2];
  const S nn = dsqrt(gw[0] * gw[0] + gw[1] * gw[1] + gw[2] * gw[2]);
  if (!(val(nn) > 0.0)) return false;
  for (int r = 0; r < 3; ++r) n[r] = gw[r] / nn;
  return true;
}

extern "C" {

// ---------------------------------------------------------------------------
// Pre-filter (Sec. 3.2): alpha_max = Eq. 1 at (f_max, f_min).  keep[k] = 1 iff
// alpha_max >= T_f (PURE: every tet kept).  amb[k] = 1 iff alpha_max lies within
// band*T_f of T_f.  Returns the number kept, or -1 on an index outside [0, N).
// ---------------------------------------------------------------------------
int64_t orc_prefilter(int64_t K, const int32_t* T, int64_t N, const float* f,
                      const OrcParams* p, int8_t* keep, int8_t* amb, double* amax_out) {
  int64_t n = 0;
  for (int64_t k = 0; k < K; ++k) {
    double fmax = -INFINITY, fmin = INFINITY;
    for (int j = 0; j < 4; ++j) {
      int32_t id = T[4 * k + j];
      if (id < 0 || id >= N) return -1;
      fmax = std::max(fmax, (double)f[id]);
      fmin = std::min(fmin, (double)f[id]);
    }
    double am = opacity_eq1<double>(fmax, fmin, p->s);
    if (amax_out) amax_out[k] = am;
    bool kp = (p->flags & ORC_PURE) ? true : (am >= p->prefilter_thresh);
    keep[k] = kp ? 1 : 0;
    amb[k] = (!(p->flags & ORC_PURE) &&
              std::fabs(am - p->prefilter_thresh) <= p->band * p->prefilter_thresh) ? 1 : 0;
    n += kp;
  }
  return n;
}

// ---------------------------------------------------------------------------
// Binning key path, an exact FP32 op sequence (compile without contraction):
//   x = fma(R0, vx, fma(R1, vy, fma(R2, vz, t0)))       (same for y, z)
//   cull if any z < znear
//   zbar = ((za + zb) + (zc + zd)) * 0.25
//   u = fma(fx, x / z, cx), v = fma(fy, y / z, cy)       (correctly rounded /)
//   i0 = max(ceil(umin - 0.5), 0), i1 = min(floor(umax - 0.5), W - 1)   (same j)
//   empty (culled) if i0 > i1 or j0 > j1
//   tile rect = [i0 / B, i1 / B] x [j0 / B, j1 / B]
// rect[4s] = (i0, i1, j0, j1) or (-1,-1,-1,-1) when culled; zbits[s] = bits of
// zbar; ntl[s] = tiles overlapped.  Returns the total number of keys.
//
// With hull != 0 (the tile test against the projected tet, Sec. 3.3
// culling): the projection of a tet is the convex hull of its projected
// vertices, so a pixel centre outside it meets no chord.  A tile of the rect
// keeps its key unless, for some edge of that hull, the four corner pixel
// centres of (tile x bbox) all lie strictly outside it.  FP32, in this order:
// for the edge (a, b) and a point p,
//   ex = bu - au, ey = bv - av,
//   E = fma(ex, pv - av, -(ey * (pu - au))),
// (a, b) is a hull edge iff E has the same nonzero sign at the other two
// vertices, and a corner is outside iff its E has the opposite strict sign.
// One-tile rects and rects wider or taller than 2 tiles keep every tile.  keep[s] (nullable)
// receives the kept cells as bits cy * ntx + cx (all ones when not tested).
// ---------------------------------------------------------------------------
static float hull_edge_fn(float au, float av, float ex, float ey, float px, float py) {
  return std::fma(ex, py - av, -(ey * (px - au)));
}

static uint32_t hull_keep_mask(const float pu[4], const float pv[4], int i0, int i1, int j0, int j1,
                               int tile) {
  const int tx0 = i0 / tile, tx1 = i1 / tile, ty0 = j0 / tile, ty1 = j1 / tile;
  const int ntx = tx1 - tx0 + 1, nty = ty1 - ty0 + 1, nt = ntx * nty;
  // one-tile rects and rects wider or taller than 2 tiles are not tested
  if (nt == 1 || ntx > 2 || nty > 2) return 0xffffffffu;
  uint32_t keep = (nt == 32) ? 0xffffffffu : ((1u << nt) - 1u);
  static const int pairs[6][4] = {{0, 1, 2, 3}, {0, 2, 1, 3}, {0, 3, 1, 2},
                                  {1, 2, 0, 3}, {1, 3, 0, 2}, {2, 3, 0, 1}};
  for (const auto& pr : pairs) {
    const int a = pr[0], b = pr[1], c = pr[2], d = pr[3];
    const float ex = pu[b] - pu[a], ey = pv[b] - pv[a];
    const float ec = hull_edge_fn(pu[a], pv[a], ex, ey, pu[c], pv[c]);
    const float ed = hull_edge_fn(pu[a], pv[a], ex, ey, pu[d], pv[d]);
    if (!((ec > 0.f && ed > 0.f) || (ec < 0.f && ed < 0.f))) continue;   // not a hull edge
    const bool pos = ec > 0.f;
    for (int cell = 0; cell < nt; ++cell) {
      if (!((keep >> cell) & 1u)) continue;
      const int tx = tx0 + cell % ntx, ty = ty0 + cell / ntx;
      const float x0 = (float)std::max(tx * tile, i0) + 0.5f;
      const float x1 = (float)std::min(tx * tile + tile - 1, i1) + 0.5f;
      const float y0 = (float)std::max(ty * tile, j0) + 0.5f;
      const float y1 = (float)std::min(ty * tile + tile - 1, j1) + 0.5f;
      const float cs[4] = {hull_edge_fn(pu[a], pv[a], ex, ey, x0, y0),
                           hull_edge_fn(pu[a], pv[a], ex, ey, x1, y0),
                           hull_edge_fn(pu[a], pv[a], ex, ey, x0, y1),
                           hull_edge_fn(pu[a], pv[a], ex, ey, x1, y1)};
      bool out = true;
      for (const float e : cs) out = out && (pos ? (e < 0.f) : (e > 0.f));
      if (out) keep &= ~(1u << cell);
    }
  }
  return keep;
}

int64_t orc_bin_prepare(int64_t ns, const int32_t* surv, const int32_t* T, const float* V,
                        const OrcCam* cam, int32_t tile, int32_t* rect, uint32_t* zbits,
                        int32_t* ntl, int32_t hull, uint32_t* keep) {
  const OrcCam& c = *cam;
  int64_t total = 0;
  const float W1 = (float)(c.width - 1), H1 = (float)(c.height - 1);
  for (int64_t s = 0; s < ns; ++s) {
    const int32_t* t = T + 4 * (int64_t)surv[s];
    float x[4], y[4], z[4];
    bool cull = false;
    for (int j = 0; j < 4; ++j) {
      const float* v = V + 3 * (int64_t)t[j];
      x[j] = std::fma(c.R[0], v[0], std::fma(c.R[1], v[1], std::fma(c.R[2], v[2], c.t[0])));
      y[j] = std::fma(c.R[3], v[0], std::fma(c.R[4], v[1], std::fma(c.R[5], v[2], c.t[1])));
      z[j] = std::fma(c.R[6], v[0], std::fma(c.R[7], v[1], std::fma(c.R[8], v[2], c.t[2])));
      if (!(z[j] >= c.znear)) cull = true;
    }
    float zb = ((z[0] + z[1]) + (z[2] + z[3])) * 0.25f;
    uint32_t zbit;
    std::memcpy(&zbit, &zb, 4);
    zbits[s] = zbit;
    rect[4 * s + 0] = rect[4 * s + 1] = rect[4 * s + 2] = rect[4 * s + 3] = -1;
    ntl[s] = 0;
    if (cull) continue;
    float umin = INFINITY, umax = -INFINITY, vmin = INFINITY, vmax = -INFINITY;
    float pu[4], pv[4];
    for (int j = 0; j < 4; ++j) {
      float u = std::fma(c.fx, x[j] / z[j], c.cx);
      float v = std::fma(c.fy, y[j] / z[j], c.cy);
      pu[j] = u;
      pv[j] = v;
      umin = std::fmin(umin, u); umax = std::fmax(umax, u);
      vmin = std::fmin(vmin, v); vmax = std::fmax(vmax, v);
    }
    float i0 = std::fmax(std::ceil(umin - 0.5f), 0.0f);
    float i1 = std::fmin(std::floor(umax - 0.5f), W1);
    float j0 = std::fmax(std::ceil(vmin - 0.5f), 0.0f);
    float j1 = std::fmin(std::floor(vmax - 0.5f), H1);
    if (!(i0 <= i1) || !(j0 <= j1)) continue;
    int ii0 = (int)i0, ii1 = (int)i1, jj0 = (int)j0, jj1 = (int)j1;
    int nt = (ii1 / tile - ii0 / tile + 1) * (jj1 / tile - jj0 / tile + 1);
    uint32_t km = 0xffffffffu;
    if (hull) {
      km = hull_keep_mask(pu, pv, ii0, ii1, jj0, jj1, tile);
      if (km != 0xffffffffu) nt = __builtin_popcount(km);   // a tested rect
      if (nt == 0) continue;      // no pixel centre of the bbox inside the hull
    }
    if (keep) keep[s] = km;
    rect[4 * s + 0] = ii0; rect[4 * s + 1] = ii1; rect[4 * s + 2] = jj0; rect[4 * s + 3] = jj1;
    ntl[s] = nt;
    total += nt;
  }
  return total;
}

// Duplicate and sort: one entry (tile, zbits, survivor index) per overlapped
// tile, sorted by (tile, zbits) with std::stable_sort (ties keep survivor
// order).  ranges[2*tile] = [start, end).
int64_t orc_bin_sort(int64_t ns, const int32_t* rect, const uint32_t* zbits, const OrcCam* cam,
                     int32_t tile, int32_t* out_tile, uint32_t* out_z, int32_t* out_val,
                     int32_t* ranges, const uint32_t* keep) {
  const int tx = (cam->width + tile - 1) / tile, ty = (cam->height + tile - 1) / tile;
  struct E { int32_t tile; uint32_t z; int32_t val; };
  std::vector<E> ent;
  for (int64_t s = 0; s < ns; ++s) {
    if (rect[4 * s] < 0) continue;
    const int a0 = rect[4 * s] / tile, a1 = rect[4 * s + 1] / tile;
    const int b0 = rect[4 * s + 2] / tile, b1 = rect[4 * s + 3] / tile;
    const int ncell = (a1 - a0 + 1) * (b1 - b0 + 1);
    for (int b = b0; b <= b1; ++b)
      for (int a = a0; a <= a1; ++a) {
        const int cell = (b - b0) * (a1 - a0 + 1) + (a - a0);
        if (keep && keep[s] != 0xffffffffu && !((keep[s] >> cell) & 1u)) continue;   // hull test
        ent.push_back({b * tx + a, zbits[s], (int32_t)s});
      }
  }
  std::stable_sort(ent.begin(), ent.end(), [](const E& p, const E& q) {
    if (p.tile != q.tile) return p.tile < q.tile;
    return p.z < q.z;
  });
  for (int i = 0; i < tx * ty; ++i) ranges[2 * i] = ranges[2 * i + 1] = 0;
  for (size_t i = 0; i < ent.size(); ++i) {
    out_tile[i] = ent[i].tile;
    out_z[i] = ent[i].z;
    out_val[i] = ent[i].val;
    if (i == 0 || ent[i - 1].tile != ent[i].tile) ranges[2 * ent[i].tile] = (int32_t)i;
    ranges[2 * ent[i].tile + 1] = (int32_t)(i + 1);
  }
  return (int64_t)ent.size();
}

// single-fragment probe (tests): camera-space vertices X (12), F (4)
int orc_fragment(const double* X, const double* F, double px, double py, double fx, double fy,
                 double cx, double cy, double s, double* out /* f_prev f_next z_in z_out alpha */) {
  double Xa[4][3], Fa[4];
  for (int j = 0; j < 4; ++j) { for (int r = 0; r < 3; ++r) Xa[j][r] = X[3 * j + r]; Fa[j] = F[j]; }
  FragOut<double> o;
  if (!eval_fragment<double>(Xa, Fa, px, py, fx, fy, cx, cy, &o)) return 0;
  out[0] = o.f_prev; out[1] = o.f_next; out[2] = o.z_in; out[3] = o.z_out;
  out[4] = opacity_eq1<double>(o.f_prev, o.f_next, s);
  return 1;
}

// gradient of the single-fragment alpha wrt X (12) and F (4), by dual numbers
int orc_fragment_grad(const double* X, const double* F, double px, double py, double fx, double fy,
                      double cx, double cy, double s, double* alpha, double* grad16) {
  typedef Dual<16> D;
  D Xa[4][3], Fa[4];
  for (int j = 0; j < 4; ++j) {
    for (int r = 0; r < 3; ++r) { Xa[j][r] = D(X[3 * j + r]); Xa[j][r].d[3 * j + r] = 1.0; }
    Fa[j] = D(F[j]); Fa[j].d[12 + j] = 1.0;
  }
  FragOut<D> o;
  if (!eval_fragment<D>(Xa, Fa, px, py, fx, fy, cx, cy, &o)) return 0;
  D a = opacity_eq1<D>(o.f_prev, o.f_next, s);
  *alpha = a.v;
  for (int i = 0; i < 16; ++i) grad16[i] = a.d[i];
  return 1;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// per-pixel compositing (Eq. 2 with the 3DGS conventions)
// ---------------------------------------------------------------------------
namespace {

struct Frag {
  int32_t s;       // survivor index
  double alpha;    // Eq. 1
  double zbar;     // mean vertex depth (Eq. 2 depth term)
  double c[3];     // tet colour: mean of the vertex colours
  double zin;      // depth of the chord's entry point (App. A.2 z_p of the nearest hit)
  double n[3];     // world-space unit normal (Eq. 2 normal term)
};

struct Blended {
  int32_t s;
  double a, T, zbar, c[3], n[3];
  bool clamped;
};

struct PixelResult {
  double C[3], D, O, N[3];
  int amb;            // ambiguous decisions met on the primary branch
  int first_amb;      // decision index of the first one (-1 none)
  std::vector<Blended> blended;
};

// Walk the fragment list.  Decision indices count every threshold test in
// the order a walk meets them (none past the stop); flip = index of the
// decision to invert (-1: none).
// Resort window (Sec. 3.3): fragments that pass the cap and skip tests enter
// a window kept sorted by the entry depth z_in (ties: earlier first); when it
// holds more than N_w fragments the nearest one leaves it and is blended; at
// the end of the list the rest leave in depth order.  N_w = 0 keeps the tile
// order; N_w < 0 sorts the whole pixel list by z_in.
struct Staged {
  Frag f;
  double a;
  bool clamped;
  bool cap_exact;   // clamped by an unambiguous cap decision: alpha' is the FP32 cap exactly
};

// The stop test of a fragment whose alpha' is the cap, after blended
// fragments that all were (n_capped of them): T (1 - alpha') is then a product
// of FP32 factors (1 - cap) and 1, which the kernel forms in FP32 (3DGS
// evaluates this test in FP32 too).  For up to three factors every order of
// the products rounds to the same FP32 value, so the decision is taken here
// in FP32 exactly, as the kernel takes it, and is not ambiguous.  With the
// 3DGS constants two capped fragments land on the threshold in real
// arithmetic: (1 - 0.99)^2 = 1e-4.
// Applies when cap and t_eps are FP32 values (the thresholds a kernel call
// receives); with other values the FP64 decision and its band stand.
static bool fp32_thresholds(const OrcParams& p) {
  return (double)(float)p.alpha_cap == p.alpha_cap && (double)(float)p.t_eps == p.t_eps;
}
static bool capped_stop_exact(int n_capped, const Staged& st, const OrcParams& p) {
  return st.cap_exact && n_capped >= 0 && n_capped <= 2 && fp32_thresholds(p);
}

static void composite(const std::vector<Frag>& fr, const OrcParams& p, int flip, bool record,
                      PixelResult* r) {
  const bool pure = (p.flags & ORC_PURE) != 0;
  double T = 1.0, C[3] = {0, 0, 0}, D = 0, Nn[3] = {0, 0, 0};
  int dec = 0;
  r->amb = 0;
  r->first_amb = -1;
  r->blended.clear();
  auto decide = [&](bool outcome, double x, double thr) {
    int id = dec++;
    if (std::fabs(x - thr) <= p.band * thr) {
      if (r->first_amb < 0) r->first_amb = id;
      r->amb++;
    }
    return (id == flip) ? !outcome : outcome;
  };
  float T32 = 1.0f;   // T as the kernel holds it, while n_capped >= 0
  int n_capped = 0;   // blended fragments so far, all exactly at the cap (-1: not so)
  // Blends one fragment (Eq. 2) unless the stop test ends the pixel first;
  // returns true when the pixel stops.
  auto emit = [&](const Staged& st) {
    const Frag& f = st.f;
    const double a = st.a;
    const double Tn = T * (1.0 - a);
    if (!pure) {
      if (capped_stop_exact(n_capped, st, p)) {
        const float Tn32 = T32 * (1.0f - (float)p.alpha_cap);
        const int id = dec++;
        const bool stop = Tn32 < (float)p.t_eps;
        if ((id == flip) ? !stop : stop) return true;
      } else if (decide(Tn < p.t_eps, Tn, p.t_eps)) {
        return true;
      }
    }
    if (st.cap_exact && n_capped >= 0) {
      T32 = T32 * (1.0f - (float)p.alpha_cap);
      ++n_capped;
    } else {
      n_capped = -1;
    }
    for (int q = 0; q < 3; ++q) C[q] += T * a * f.c[q];
    for (int q = 0; q < 3; ++q) Nn[q] += T * a * f.n[q];
    D += T * a * f.zbar;
    if (record)
      r->blended.push_back({f.s, a, T, f.zbar, {f.c[0], f.c[1], f.c[2]}, {f.n[0], f.n[1], f.n[2]},
                            st.clamped});
    T = Tn;
    return false;
  };
  auto near_tie = [&](double x, double y) {
    return std::fabs(x - y) <= 1e-5 * std::max(std::fabs(x), std::fabs(y));
  };
  // One pass in list order, as a walk that stops meets the fragments: the cap
  // and skip decisions of each fragment, its way through the window (if any)
  // and the stop test of each fragment leaving it.  Decisions past the stop
  // are never taken.
  const size_t wcap = (p.window < 0) ? fr.size() + 1 : (size_t)p.window;
  std::vector<Staged> win;
  bool stopped = false;
  for (const Frag& f : fr) {
    double a = f.alpha;
    bool clamped = false, cap_exact = false;
    if (!pure) {
      const int amb0 = r->amb;
      if (decide(a > p.alpha_cap, a, p.alpha_cap)) {
        a = p.alpha_cap;
        clamped = true;
        cap_exact = r->amb == amb0;
      }
      if (decide(a < p.alpha_skip, a, p.alpha_skip)) continue;
    } else if (!(a > 0.0)) {
      continue;
    }
    const Staged st = {f, a, clamped, cap_exact};
    if (p.window == 0) {
      if (emit(st)) { stopped = true; break; }
      continue;
    }
    size_t pos = 0;
    while (pos < win.size() && win[pos].f.zin <= st.f.zin) ++pos;
    for (const Staged& w : win)
      if (near_tie(w.f.zin, st.f.zin)) r->amb += 2;  // order not decidable in FP32
    win.insert(win.begin() + pos, st);
    if (win.size() > wcap) {
      const Staged w = win.front();
      win.erase(win.begin());
      if (emit(w)) { stopped = true; break; }
    }
  }
  if (!stopped)
    for (const Staged& w : win)
      if (emit(w)) break;
  for (int q = 0; q < 3; ++q) r->C[q] = C[q];
  for (int q = 0; q < 3; ++q) r->N[q] = Nn[q];
  r->D = D;
  r->O = 1.0 - T;
}

}  // namespace

extern "C" {

// ---------------------------------------------------------------------------
// Render one view.  Inputs: the survivor list (original tet ids), the binning
// result of orc_bin_prepare/orc_bin_sort.  Outputs (planar, H x W):
//   img (3HW), alpha (HW), depth (HW): primary branch
//   amb (HW): ambiguous decisions on the primary branch
//   alt_img/alt_alpha/alt_depth: first ambiguous decision inverted (== primary
//   when amb == 0)
//   nfrag (HW): fragments (hits) met by the walk before it stopped
// When dimg != nullptr, also accumulates the gradient of
//   L = sum(dimg * img) + sum(dalpha * alpha) + sum(ddepth * depth)
// into dV (3N), df (N), drgb (3N) (FP64, added to what is there).
// branch (HW, nullable): 1 differentiates the pixel's alternative branch (its
// first ambiguous decision inverted) instead of the primary one.
// dV_abs, df_abs, drgb_abs (nullable): the sums of the absolute values of the
// per-fragment terms added into each gradient entry (the scale of the
// rounding a sum of those terms in another order can show).
// dV_kink, df_kink (nullable): per entry, the sum over fragments whose ray
// passes within 1e-4 (relative depth) of an edge of its entry or exit face of
// the largest change of that fragment's term when another face nearly as
// near gives the entry or exit point (the other one-sided derivative at the
// chord's kink, which a computation in another precision may take).
// dV_graze (nullable): per entry, the sum over the fragments of its tet of
// (the largest of the fragment's terms through its opacity over the tet's
// four vertices) / c^2, c the smaller of |cos| of the angles between the
// pixel ray and the normals of the chord's entry and exit faces (a face seen
// at grazing incidence makes the entry or exit point, and most of all its
// derivative, ill-conditioned: in a precision with unit roundoff u the
// rounding error of the terms grows as about u / c^2 times their largest,
// and it reaches every vertex through the face planes they share).
// ---------------------------------------------------------------------------
int orc_render(int64_t N, const float* V, const float* f, const float* rgb, const int32_t* T,
               int64_t ns, const int32_t* surv, const int32_t* rect, const OrcCam* cam,
               const OrcParams* p, const int32_t* key_val, const int32_t* ranges,
               double* img, double* alpha, double* depth, int32_t* amb,
               double* alt_img, double* alt_alpha, double* alt_depth, int32_t* nfrag,
               const float* dimg, const float* dalpha, const float* ddepth,
               double* dV, double* df, double* drgb, int nthreads,
               const double* V64, const double* f64, const double* rgb64,
               double* nrm, double* alt_nrm, const float* dnrm, const int8_t* branch,
               double* dV_abs, double* df_abs, double* drgb_abs, double* dV_kink,
               double* df_kink, double* dV_graze, int32_t* nblend, int32_t* blend_slots,
               int blend_cap) {
  const OrcCam& c = *cam;
  const Fields fld(N, V, f, rgb, V64, f64, rgb64);
  const int W = c.width, H = c.height, B = p->tile;
  const int tx = (W + B - 1) / B;
  const bool want_grad = dimg != nullptr;
  const int64_t HW = (int64_t)H * W;
  // nthreads > 0 caps this call's team only (no process-wide setting)
#ifdef _OPENMP
  const int nth = (nthreads > 0) ? nthreads : omp_get_max_threads();
#else
  const int nth = 1;
#endif
  (void)nth;

#pragma omp parallel for schedule(dynamic, 1) num_threads(nth)
  for (int j = 0; j < H; ++j) {
    std::vector<Frag> fr;
    PixelResult pr, alt;
    for (int i = 0; i < W; ++i) {
      const int tile = (j / B) * tx + (i / B);
      const double px = i + 0.5, py = j + 0.5;
      fr.clear();
      // walk this tile's list in key order; the pixel-local fragments
      struct FragG { double g[16]; };
      std::vector<FragG> fgrad;
      int hits = 0;
      for (int e = ranges[2 * tile]; e < ranges[2 * tile + 1]; ++e) {
        const int32_t s = key_val[e];
        const int32_t* r4 = rect + 4 * (int64_t)s;
        if (i < r4[0] || i > r4[1] || j < r4[2] || j > r4[3]) continue;
        const int32_t* t = T + 4 * (int64_t)surv[s];
        double X[4][3], F[4];
        for (int q = 0; q < 4; ++q) { cam_xform(c, &fld.V[3 * (int64_t)t[q]], X[q]); F[q] = fld.f[t[q]]; }
        Frag fg;
        fg.s = s;
        FragOut<double> o;
        if (!eval_fragment<double>(X, F, px, py, c.fx, c.fy, c.cx, c.cy, &o)) continue;
        ++hits;
        fg.zin = o.z_in;
        fg.alpha = opacity_eq1<double>(o.f_prev, o.f_next, p->s);
        fg.zbar = 0.25 * (X[0][2] + X[1][2] + X[2][2] + X[3][2]);
        if (!tet_normal_world<double>(X, F, c, fg.n)) fg.n[0] = fg.n[1] = fg.n[2] = 0.0;
        for (int q = 0; q < 3; ++q)
          fg.c[q] = 0.25 * (((fld.rgb[3 * t[0] + q] + fld.rgb[3 * t[1] + q]) + fld.rgb[3 * t[2] + q]) + fld.rgb[3 * t[3] + q]);
        fr.push_back(fg);
      }
      composite(fr, *p, -1, want_grad || nblend != nullptr, &pr);
      const int64_t pix = (int64_t)j * W + i;
      if (nblend) {
        // the pixel's blended fragments: how many, and the view slots of the
        // first blend_cap of them in blend order
        nblend[pix] = (int32_t)pr.blended.size();
        for (int q = 0; q < blend_cap && q < (int)pr.blended.size(); ++q)
          blend_slots[pix * blend_cap + q] = pr.blended[q].s;
      }
      for (int q = 0; q < 3; ++q) img[q * HW + pix] = pr.C[q];
      if (nrm)
        for (int q = 0; q < 3; ++q) nrm[q * HW + pix] = pr.N[q];
      alpha[pix] = pr.O;
      depth[pix] = pr.D;
      amb[pix] = pr.amb;
      nfrag[pix] = hits;
      const bool use_alt = want_grad && branch && branch[(int64_t)j * W + i] && pr.first_amb >= 0;
      if (pr.first_amb >= 0) {
        composite(fr, *p, pr.first_amb, use_alt, &alt);
        for (int q = 0; q < 3; ++q) alt_img[q * HW + pix] = alt.C[q];
        if (alt_nrm)
          for (int q = 0; q < 3; ++q) alt_nrm[q * HW + pix] = alt.N[q];
        alt_alpha[pix] = alt.O;
        alt_depth[pix] = alt.D;
      } else {
        for (int q = 0; q < 3; ++q) alt_img[q * HW + pix] = pr.C[q];
        if (alt_nrm)
          for (int q = 0; q < 3; ++q) alt_nrm[q * HW + pix] = pr.N[q];
        alt_alpha[pix] = pr.O;
        alt_depth[pix] = pr.D;
      }
      // ---- adjoint of the composite (the primary branch, or the alternative) ----
      const PixelResult& ad = use_alt ? alt : pr;
      if (!want_grad || ad.blended.empty()) continue;
      const double gC[3] = {dimg[pix], dimg[HW + pix], dimg[2 * HW + pix]};
      const double gO = dalpha[pix], gD = ddepth[pix];
      const double gN[3] = {dnrm ? (double)dnrm[pix] : 0.0, dnrm ? (double)dnrm[HW + pix] : 0.0,
                            dnrm ? (double)dnrm[2 * HW + pix] : 0.0};
      const double Tfin = 1.0 - ad.O;
      double Ssuf = 0.0;
      for (int b = (int)ad.blended.size() - 1; b >= 0; --b) {
        const Blended& bl = ad.blended[b];
        const double w = gC[0] * bl.c[0] + gC[1] * bl.c[1] + gC[2] * bl.c[2] + gD * bl.zbar +
                         gN[0] * bl.n[0] + gN[1] * bl.n[1] + gN[2] * bl.n[2];
        const double dLda = bl.T * w - (Ssuf - gO * Tfin) / (1.0 - bl.a);
        Ssuf += bl.T * bl.a * w;
        const int32_t* t = T + 4 * (int64_t)surv[bl.s];
        // colour: c = mean of the 4 vertex colours
        for (int q = 0; q < 4; ++q)
          for (int ch = 0; ch < 3; ++ch) {
#pragma omp atomic
            drgb[3 * (size_t)t[q] + ch] += 0.25 * bl.T * bl.a * gC[ch];
            if (drgb_abs) {
#pragma omp atomic
              drgb_abs[3 * (size_t)t[q] + ch] += std::fabs(0.25 * bl.T * bl.a * gC[ch]);
            }
          }
        // depth term: zbar = mean camera z -> world via R^T (third row)
        double dX[4][3] = {{0}};
        const double dz = 0.25 * bl.T * bl.a * gD;
        for (int q = 0; q < 4; ++q) dX[q][2] += dz;
        double dF[4] = {0, 0, 0, 0};
        if (!bl.clamped && dLda != 0.0) {
          typedef Dual<16> D16;
          D16 X[4][3], F[4];
          for (int q = 0; q < 4; ++q) {
            double xd[3];
            cam_xform(c, &fld.V[3 * (int64_t)t[q]], xd);
            for (int r = 0; r < 3; ++r) { X[q][r] = D16(xd[r]); X[q][r].d[3 * q + r] = 1.0; }
            F[q] = D16(fld.f[t[q]]);
            F[q].d[12 + q] = 1.0;
          }
          FragOut<D16> o;
          if (eval_fragment<D16>(X, F, px, py, c.fx, c.fy, c.cx, c.cy, &o)) {
            D16 a = opacity_eq1<D16>(o.f_prev, o.f_next, p->s);
            for (int q = 0; q < 4; ++q) {
              for (int r = 0; r < 3; ++r) dX[q][r] += dLda * a.d[3 * q + r];
              dF[q] += dLda * a.d[12 + q];
            }
            if (dV_graze) {
              // grazing cosines of the entry and exit faces for this ray
              const double ray[3] = {(px - c.cx) / c.fx, (py - c.cy) / c.fy, 1.0};
              const double rl = std::sqrt(ray[0] * ray[0] + ray[1] * ray[1] + 1.0);
              double cmin = 1.0;
              for (const int k : {o.k_in, o.k_out}) {
                const int ia = kFaces[k][0], ib = kFaces[k][1], ic = kFaces[k][2];
                double e1[3], e2[3];
                for (int r = 0; r < 3; ++r) {
                  e1[r] = val(X[ib][r]) - val(X[ia][r]);
                  e2[r] = val(X[ic][r]) - val(X[ia][r]);
                }
                const double nx = e1[1] * e2[2] - e1[2] * e2[1], ny = e1[2] * e2[0] - e1[0] * e2[2],
                             nz = e1[0] * e2[1] - e1[1] * e2[0];
                const double nl = std::sqrt(nx * nx + ny * ny + nz * nz);
                if (nl > 0.0)
                  cmin = std::min(cmin, std::fabs(nx * ray[0] + ny * ray[1] + nz * ray[2]) / (nl * rl));
              }
              // the fragment's largest term (world components bounded through
              // |R^T|): rounding of the shared record-field gradients reaches
              // every vertex of the tet at that scale
              const double wgt = 1.0 / std::max(cmin * cmin, 1e-12);
              double gmax = 0.0;
              for (int q = 0; q < 4; ++q)
                for (int r = 0; r < 3; ++r) {
                  double g = 0.0;
                  for (int k = 0; k < 3; ++k) g += std::fabs(c.R[3 * k + r]) * std::fabs(dLda * a.d[3 * q + k]);
                  gmax = std::max(gmax, g);
                }
              for (int q = 0; q < 4; ++q)
                for (int r = 0; r < 3; ++r) {
#pragma omp atomic
                  dV_graze[3 * (size_t)t[q] + r] += wgt * gmax;
                }
            }
            if (dV_kink && df_kink) {
              int ai[4], ao[4], ni = 0, no = 0;
              near_kink_faces<D16>(X, F, px, py, c.fx, c.fy, c.cx, c.cy, o, 1e-4, 1e-4, ai, &ni,
                                   ao, &no);
              if (ni + no > 0) {
                FaceEval<D16> fe[4];
                eval_faces<D16>(X, F, px, py, c.fx, c.fy, c.cx, c.cy, fe);
                int cin[5] = {o.k_in}, cout_[5] = {o.k_out};
                for (int k = 0; k < ni; ++k) cin[k + 1] = ai[k];
                for (int k = 0; k < no; ++k) cout_[k + 1] = ao[k];
                double dmax[16] = {0};
                for (int x = 0; x <= ni; ++x)
                  for (int y = 0; y <= no; ++y) {
                    if ((x == 0 && y == 0) || cin[x] == cout_[y]) continue;
                    const D16 a2 = opacity_eq1<D16>(fe[cin[x]].f, fe[cout_[y]].f, p->s);
                    for (int k = 0; k < 16; ++k)
                      dmax[k] = std::max(dmax[k], std::fabs(dLda * (a2.d[k] - a.d[k])));
                  }
                for (int q = 0; q < 4; ++q) {
                  for (int r = 0; r < 3; ++r) {
                    // |R^T d| <= sum_k |R_kr| |d_k| per world component
                    const double b = std::fabs(c.R[r]) * dmax[3 * q] +
                                     std::fabs(c.R[3 + r]) * dmax[3 * q + 1] +
                                     std::fabs(c.R[6 + r]) * dmax[3 * q + 2];
#pragma omp atomic
                    dV_kink[3 * (size_t)t[q] + r] += b;
                  }
#pragma omp atomic
                  df_kink[t[q]] += dmax[12 + q];
                }
              }
            }
          }
        }
        if (dnrm && (gN[0] != 0.0 || gN[1] != 0.0 || gN[2] != 0.0)) {
          // normal term: dL/dn = T a gN through n = g_w / |g_w| (App. A.3)
          typedef Dual<16> D16;
          D16 X[4][3], F[4], nd[3];
          for (int q = 0; q < 4; ++q) {
            double xd[3];
            cam_xform(c, &fld.V[3 * (int64_t)t[q]], xd);
            for (int r = 0; r < 3; ++r) { X[q][r] = D16(xd[r]); X[q][r].d[3 * q + r] = 1.0; }
            F[q] = D16(fld.f[t[q]]);
            F[q].d[12 + q] = 1.0;
          }
          if (tet_normal_world<D16>(X, F, c, nd)) {
            const double wgt = bl.T * bl.a;
            for (int r = 0; r < 3; ++r) {
              const double gn = wgt * gN[r];
              for (int q = 0; q < 4; ++q) {
                for (int k = 0; k < 3; ++k) dX[q][k] += gn * nd[r].d[3 * q + k];
                dF[q] += gn * nd[r].d[12 + q];
              }
            }
          }
        }
        for (int q = 0; q < 4; ++q) {
          // world gradient: x_c = R v + t  ->  dv = R^T dx_c
          for (int r = 0; r < 3; ++r) {
            double g = c.R[r] * dX[q][0] + c.R[3 + r] * dX[q][1] + c.R[6 + r] * dX[q][2];
#pragma omp atomic
            dV[3 * (size_t)t[q] + r] += g;
            if (dV_abs) {
#pragma omp atomic
              dV_abs[3 * (size_t)t[q] + r] += std::fabs(g);
            }
          }
#pragma omp atomic
          df[t[q]] += dF[q];
          if (df_abs) {
#pragma omp atomic
            df_abs[t[q]] += std::fabs(dF[q]);
          }
        }
      }
    }
  }
  return 0;
}

// ---------------------------------------------------------------------------
// Directional derivative of L along (tV, tf, trgb) by a single-tangent dual
// pass through the whole render (tests: pins the adjoint).  Uses the same
// binning lists; returns L in out[0] and dL in out[1].
// ---------------------------------------------------------------------------
int orc_render_dirderiv(int64_t N, const float* V, const float* f, const float* rgb,
                        const int32_t* T, int64_t ns, const int32_t* surv, const int32_t* rect,
                        const OrcCam* cam, const OrcParams* p, const int32_t* key_val,
                        const int32_t* ranges, const float* dimg, const float* dalpha,
                        const float* ddepth, const double* tV, const double* tf,
                        const double* trgb, double* out, const double* V64, const double* f64,
                        const double* rgb64, const float* dnrm) {
  typedef Dual<1> D1;
  const OrcCam& c = *cam;
  const Fields fld(N, V, f, rgb, V64, f64, rgb64);
  const int W = c.width, H = c.height, B = p->tile;
  const int tx = (W + B - 1) / B;
  const bool pure = (p->flags & ORC_PURE) != 0;
  const int64_t HW = (int64_t)H * W;
  D1 L(0.0);
  (void)ns;
  for (int j = 0; j < H; ++j)
    for (int i = 0; i < W; ++i) {
      const int tile = (j / B) * tx + (i / B);
      const double px = i + 0.5, py = j + 0.5;
      D1 Tr(1.0), C[3] = {D1(0.0), D1(0.0), D1(0.0)}, Dp(0.0), Nn[3] = {D1(0.0), D1(0.0), D1(0.0)};
      struct FD { D1 a, zb, cc[3], nn[3]; double zin; };
      std::vector<FD> in;
      for (int e = ranges[2 * tile]; e < ranges[2 * tile + 1]; ++e) {
        const int32_t s = key_val[e];
        const int32_t* r4 = rect + 4 * (int64_t)s;
        if (i < r4[0] || i > r4[1] || j < r4[2] || j > r4[3]) continue;
        const int32_t* t = T + 4 * (int64_t)surv[s];
        D1 X[4][3], F[4];
        for (int q = 0; q < 4; ++q) {
          const double* v = &fld.V[3 * (int64_t)t[q]];
          for (int r = 0; r < 3; ++r) {
            double xv = (double)c.R[3 * r] * v[0] + (double)c.R[3 * r + 1] * v[1] +
                        (double)c.R[3 * r + 2] * v[2] + (double)c.t[r];
            double xt = (double)c.R[3 * r] * tV[3 * t[q]] + (double)c.R[3 * r + 1] * tV[3 * t[q] + 1] +
                        (double)c.R[3 * r + 2] * tV[3 * t[q] + 2];
            X[q][r] = D1(xv);
            X[q][r].d[0] = xt;
          }
          F[q] = D1(fld.f[t[q]]);
          F[q].d[0] = tf[t[q]];
        }
        FragOut<D1> o;
        if (!eval_fragment<D1>(X, F, px, py, c.fx, c.fy, c.cx, c.cy, &o)) continue;
        D1 a = opacity_eq1<D1>(o.f_prev, o.f_next, p->s);
        if (!pure) {
          if (a.v > p->alpha_cap) a = D1(p->alpha_cap);
          if (a.v < p->alpha_skip) continue;
        } else if (!(a.v > 0.0)) {
          continue;
        }
        FD fd;
        fd.a = a;
        fd.zin = o.z_in.v;
        if (!tet_normal_world<D1>(X, F, c, fd.nn)) fd.nn[0] = fd.nn[1] = fd.nn[2] = D1(0.0);
        fd.zb = 0.25 * (((X[0][2] + X[1][2]) + X[2][2]) + X[3][2]);
        for (int q = 0; q < 3; ++q) {
          D1 cc = 0.25 * (((D1(fld.rgb[3 * t[0] + q]) + D1(fld.rgb[3 * t[1] + q])) + D1(fld.rgb[3 * t[2] + q])) + D1(fld.rgb[3 * t[3] + q]));
          cc.d[0] = 0.25 * (trgb[3 * t[0] + q] + trgb[3 * t[1] + q] + trgb[3 * t[2] + q] + trgb[3 * t[3] + q]);
          fd.cc[q] = cc;
        }
        in.push_back(fd);
      }
      std::vector<FD> order;
      if (p->window == 0) {
        order = in;
      } else {
        const size_t cap = (p->window < 0) ? in.size() + 1 : (size_t)p->window;
        std::vector<FD> win;
        for (const FD& fd : in) {
          size_t pos = 0;
          while (pos < win.size() && win[pos].zin <= fd.zin) ++pos;
          win.insert(win.begin() + pos, fd);
          if (win.size() > cap) { order.push_back(win.front()); win.erase(win.begin()); }
        }
        for (const FD& w : win) order.push_back(w);
      }
      float T32 = 1.0f;
      int n_capped = 0;
      for (const FD& fd : order) {
        D1 Tn = Tr * (1.0 - fd.a);
        if (!pure) {
          // the stop test as in composite(): exact in FP32 after capped fragments
          const bool capped = fd.a.v == p->alpha_cap;
          if (capped && n_capped >= 0 && n_capped <= 2 && fp32_thresholds(*p)) {
            const float Tn32 = T32 * (1.0f - (float)p->alpha_cap);
            if (Tn32 < (float)p->t_eps) break;
          } else if (Tn.v < p->t_eps) {
            break;
          }
          if (capped && n_capped >= 0) {
            T32 = T32 * (1.0f - (float)p->alpha_cap);
            ++n_capped;
          } else {
            n_capped = -1;
          }
        }
        for (int q = 0; q < 3; ++q) C[q] = C[q] + Tr * fd.a * fd.cc[q];
        for (int q = 0; q < 3; ++q) Nn[q] = Nn[q] + Tr * fd.a * fd.nn[q];
        Dp = Dp + Tr * fd.a * fd.zb;
        Tr = Tn;
      }
      const int64_t pix = (int64_t)j * W + i;
      L = L + (double)dimg[pix] * C[0] + (double)dimg[HW + pix] * C[1] + (double)dimg[2 * HW + pix] * C[2] +
          (double)dalpha[pix] * (1.0 - Tr) + (double)ddepth[pix] * Dp;
      if (dnrm)
        L = L + (double)dnrm[pix] * Nn[0] + (double)dnrm[HW + pix] * Nn[1] +
            (double)dnrm[2 * HW + pix] * Nn[2];
    }
  out[0] = L.v;
  out[1] = L.d[0];
  return 0;
}

}  // extern "C"
