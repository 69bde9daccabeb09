// Oracle for the geometry-stage terms of TeT-Splatting.  TEST INFRASTRUCTURE
// ONLY: only the test suite, the smoke check and the benchmark's CPU-baseline
// leg may load this library.  It shares no code with the CUDA path.
//
//   tet_edges       the unique edges of a tetrahedral grid (each tet has six),
//                   as (lo, hi) vertex pairs sorted lexicographically.
//   regularizers    Sec. 4.2 "Eikonal loss": L_eik = sum over tets k of
//                   (|g_k| - 1)^2, with g_k the gradient of tet k's affine SDF
//                   obtained from the 4 x 4 system of App. A.3 (rows
//                   [v_i^T 1], right-hand side f_i), solved here by Gaussian
//                   elimination with partial pivoting.
//                   Sec. 4.2 "Normal consistency loss": the per-tet normals
//                   n_k = g_k / |g_k| are carried to the vertices and
//                   L_nc = sum over edges (a, b) of (1 - cos(m_a, m_b)).
//                   FP64; gradients by the hand-written adjoint (the transposed
//                   4 x 4 solve), checked against forward-mode dual numbers.
//   marching_tets   Marching Tetrahedra (Sec. 3.1, the mesh extraction the
//                   representation keeps): a vertex on every grid edge whose
//                   end points lie on different sides of the zero level set
//                   (positive: f > 0), at the zero of the linear interpolation;
//                   one triangle per tet with a 1-3 sign split and two per tet
//                   with a 2-2 split, wound so that the normal points towards
//                   increasing f.
//   survivor_bounds, fit_grid
//                   the coarse-to-fine pre-filter of App. B.1: the axis-aligned
//                   bounds of the first round's survivors, and the grid mapped
//                   per axis onto those bounds (widened by a pad fraction of
//                   their extent) for the second round.
//
// Readings where the paper is silent:
//   * "project the tet normals onto vertices": m_v = unweighted sum of the
//     unit normals of the tets that contain v;
//   * the sums run over every tet and every unique edge of the grid passed in;
//   * a tet whose 4 x 4 system is singular (flat tet) contributes to neither
//     loss; a tet with g = 0 contributes 1 to L_eik (zero gradient there) and
//     nothing to m; an edge with a zero vertex sum contributes 1 to L_nc
//     (cos taken as 0) with zero gradient.
//
//   * Marching Tetrahedra: vertices are numbered by the order of their edges
//     in the sorted unique-edge list; triangles follow the tets in order.  A
//     2-2 tet with positive local vertices p < q and negative r < s has the
//     quad (pr, ps, qs, qr) (each a crossing edge), split along pr-qs into
//     (pr, ps, qs) and (pr, qs, qr).  A 1-3 tet with odd vertex o and others
//     a < b < c gives (oa, ob, oc).  The winding is then chosen from the sign
//     of a vertex determinant (see orc_marching_tets) so that the normal
//     points towards increasing f.
//
// Parity status: pinned by closed forms (affine fields, the two-tet
// configuration, the Kuhn-grid edge count, a hand-cut single tet),
// invariances, dual numbers, finite differences, and for the extracted mesh
// by watertightness, Euler characteristic and enclosed volume.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <utility>
#include <vector>

#include "dual.h"

namespace {

// Solves M x = rhs (4 x 4, in place) by Gaussian elimination with partial
// pivoting.  Returns false when a pivot is exactly zero.
template <class S>
bool solve4(S M[4][4], S rhs[4], S x[4]) {
  int perm[4] = {0, 1, 2, 3};
  for (int col = 0; col < 4; ++col) {
    int piv = col;
    for (int r = col + 1; r < 4; ++r)
      if (std::fabs(val(M[r][col])) > std::fabs(val(M[piv][col]))) piv = r;
    if (val(M[piv][col]) == 0.0) return false;
    if (piv != col) {
      for (int k = 0; k < 4; ++k) std::swap(M[piv][k], M[col][k]);
      std::swap(rhs[piv], rhs[col]);
      std::swap(perm[piv], perm[col]);
    }
    for (int r = col + 1; r < 4; ++r) {
      const S fct = M[r][col] / M[col][col];
      for (int k = col; k < 4; ++k) M[r][k] = M[r][k] - fct * M[col][k];
      rhs[r] = rhs[r] - fct * rhs[col];
    }
  }
  for (int r = 3; r >= 0; --r) {
    S acc = rhs[r];
    for (int k = r + 1; k < 4; ++k) acc = acc - M[r][k] * x[k];
    x[r] = acc / M[r][r];
  }
  return true;
}

// App. A.3: f(x) = g . x + c through the four vertices; [v_i^T 1] [g; c] = f_i.
template <class S>
bool tet_affine(const S v[4][3], const S f[4], S g[3]) {
  S M[4][4], rhs[4], x[4];
  for (int i = 0; i < 4; ++i) {
    for (int r = 0; r < 3; ++r) M[i][r] = v[i][r];
    M[i][3] = S(1.0);
    rhs[i] = f[i];
  }
  if (!solve4(M, rhs, x)) return false;
  for (int r = 0; r < 3; ++r) g[r] = x[r];
  return true;
}

// Transposed solve for the adjoint: A^T lambda = gamma with A rows [v_i^T 1].
bool tet_affine_adjoint(const double v[4][3], const double gamma[4], double lambda[4]) {
  double M[4][4], rhs[4];
  for (int i = 0; i < 4; ++i) {
    for (int r = 0; r < 3; ++r) M[r][i] = v[i][r];
    M[3][i] = 1.0;
    rhs[i] = gamma[i];
  }
  return solve4(M, rhs, lambda);
}

// Both losses for a generic scalar type (value or dual numbers).
template <class S>
void losses(int64_t N, const S* V, int64_t K, const int32_t* T, const S* f, int64_t E,
            const int32_t* edges, S* L_eik, S* L_nc) {
  std::vector<S> m(3 * N, S(0.0));
  S le(0.0), ln(0.0);
  for (int64_t k = 0; k < K; ++k) {
    S v[4][3], fv[4], g[3];
    for (int i = 0; i < 4; ++i) {
      const int64_t id = T[4 * k + i];
      for (int r = 0; r < 3; ++r) v[i][r] = V[3 * id + r];
      fv[i] = f[id];
    }
    if (!tet_affine(v, fv, g)) continue;
    const S gn = dsqrt(g[0] * g[0] + g[1] * g[1] + g[2] * g[2]);
    le = le + (gn - 1.0) * (gn - 1.0);
    if (!(val(gn) > 0.0)) continue;
    for (int i = 0; i < 4; ++i) {
      const int64_t id = T[4 * k + i];
      for (int r = 0; r < 3; ++r) m[3 * id + r] = m[3 * id + r] + g[r] / gn;
    }
  }
  for (int64_t e = 0; e < E; ++e) {
    const int64_t a = edges[2 * e], b = edges[2 * e + 1];
    const S* ma = &m[3 * a];
    const S* mb = &m[3 * b];
    const S na = dsqrt(ma[0] * ma[0] + ma[1] * ma[1] + ma[2] * ma[2]);
    const S nb = dsqrt(mb[0] * mb[0] + mb[1] * mb[1] + mb[2] * mb[2]);
    if (val(na) > 0.0 && val(nb) > 0.0)
      ln = ln + (1.0 - (ma[0] * mb[0] + ma[1] * mb[1] + ma[2] * mb[2]) / (na * nb));
    else
      ln = ln + 1.0;
  }
  *L_eik = le;
  *L_nc = ln;
}

}  // namespace

extern "C" {

// Unique edges of the grid, sorted by (lo, hi); out holds up to 6K pairs.
// Returns the number of edges, or -1 on an index outside [0, N).
int64_t orc_tet_edges(int64_t N, int64_t K, const int32_t* T, int32_t* out) {
  std::vector<std::pair<int32_t, int32_t>> e;
  e.reserve(6 * K);
  static const int pairs[6][2] = {{0, 1}, {0, 2}, {0, 3}, {1, 2}, {1, 3}, {2, 3}};
  for (int64_t k = 0; k < K; ++k) {
    for (int i = 0; i < 4; ++i)
      if (T[4 * k + i] < 0 || T[4 * k + i] >= N) return -1;
    for (const auto& p : pairs) {
      const int32_t a = T[4 * k + p[0]], b = T[4 * k + p[1]];
      if (a != b) e.emplace_back(std::min(a, b), std::max(a, b));
    }
  }
  std::sort(e.begin(), e.end());
  e.erase(std::unique(e.begin(), e.end()), e.end());
  for (size_t i = 0; i < e.size(); ++i) {
    out[2 * i] = e[i].first;
    out[2 * i + 1] = e[i].second;
  }
  return (int64_t)e.size();
}

// L_eik and L_nc (out[0], out[1]) and, when dV / df are not null, the
// gradients of w_eik L_eik + w_nc L_nc (overwritten).
void orc_regularizers(int64_t N, const double* V, int64_t K, const int32_t* T, const double* f,
                      int64_t E, const int32_t* edges, double w_eik, double w_nc, double* out,
                      double* dV, double* df) {
  losses<double>(N, V, K, T, f, E, edges, &out[0], &out[1]);
  if (!dV || !df) return;
  // forward quantities kept for the adjoint
  std::vector<double> g(3 * K, 0.0), gn(K, 0.0), m(3 * N, 0.0);
  std::vector<char> ok(K, 0);
  for (int64_t k = 0; k < K; ++k) {
    double v[4][3], fv[4], gk[3];
    for (int i = 0; i < 4; ++i) {
      const int64_t id = T[4 * k + i];
      for (int r = 0; r < 3; ++r) v[i][r] = V[3 * id + r];
      fv[i] = f[id];
    }
    if (!tet_affine(v, fv, gk)) continue;
    ok[k] = 1;
    for (int r = 0; r < 3; ++r) g[3 * k + r] = gk[r];
    gn[k] = std::sqrt(gk[0] * gk[0] + gk[1] * gk[1] + gk[2] * gk[2]);
    if (gn[k] > 0.0)
      for (int i = 0; i < 4; ++i)
        for (int r = 0; r < 3; ++r) m[3 * T[4 * k + i] + r] += gk[r] / gn[k];
  }
  // L_nc adjoint: d(1 - cos)/d m_a = -(m_b / (|m_a||m_b|) - cos m_a / |m_a|^2)
  std::vector<double> dm(3 * N, 0.0);
  for (int64_t e = 0; e < E; ++e) {
    const int64_t a = edges[2 * e], b = edges[2 * e + 1];
    const double* ma = &m[3 * a];
    const double* mb = &m[3 * b];
    const double na = std::sqrt(ma[0] * ma[0] + ma[1] * ma[1] + ma[2] * ma[2]);
    const double nb = std::sqrt(mb[0] * mb[0] + mb[1] * mb[1] + mb[2] * mb[2]);
    if (!(na > 0.0 && nb > 0.0)) continue;
    const double cs = (ma[0] * mb[0] + ma[1] * mb[1] + ma[2] * mb[2]) / (na * nb);
    for (int r = 0; r < 3; ++r) {
      dm[3 * a + r] -= w_nc * (mb[r] / (na * nb) - cs * ma[r] / (na * na));
      dm[3 * b + r] -= w_nc * (ma[r] / (na * nb) - cs * mb[r] / (nb * nb));
    }
  }
  std::fill(dV, dV + 3 * N, 0.0);
  std::fill(df, df + N, 0.0);
  for (int64_t k = 0; k < K; ++k) {
    if (!ok[k] || !(gn[k] > 0.0)) continue;
    const double* gk = &g[3 * k];
    const double nk[3] = {gk[0] / gn[k], gk[1] / gn[k], gk[2] / gn[k]};
    double dn[3] = {0.0, 0.0, 0.0};
    for (int i = 0; i < 4; ++i)
      for (int r = 0; r < 3; ++r) dn[r] += dm[3 * T[4 * k + i] + r];
    const double ndn = nk[0] * dn[0] + nk[1] * dn[1] + nk[2] * dn[2];
    double gamma[4] = {0.0, 0.0, 0.0, 0.0};
    for (int r = 0; r < 3; ++r)
      gamma[r] = w_eik * 2.0 * (gn[k] - 1.0) * nk[r] + (dn[r] - ndn * nk[r]) / gn[k];
    double v[4][3], lambda[4];
    for (int i = 0; i < 4; ++i)
      for (int r = 0; r < 3; ++r) v[i][r] = V[3 * T[4 * k + i] + r];
    if (!tet_affine_adjoint(v, gamma, lambda)) continue;
    for (int i = 0; i < 4; ++i) {
      const int64_t id = T[4 * k + i];
      df[id] += lambda[i];
      for (int r = 0; r < 3; ++r) dV[3 * id + r] -= lambda[i] * gk[r];
    }
  }
}

// Directional derivative of w_eik L_eik + w_nc L_nc along (tV, tf) by dual
// numbers: out = (value, derivative).
void orc_regularizers_dirderiv(int64_t N, const double* V, int64_t K, const int32_t* T,
                               const double* f, int64_t E, const int32_t* edges, double w_eik,
                               double w_nc, const double* tV, const double* tf, double* out) {
  using D1 = Dual<1>;
  std::vector<D1> Vd(3 * N), fd(N);
  for (int64_t i = 0; i < 3 * N; ++i) {
    Vd[i] = D1(V[i]);
    Vd[i].d[0] = tV[i];
  }
  for (int64_t i = 0; i < N; ++i) {
    fd[i] = D1(f[i]);
    fd[i].d[0] = tf[i];
  }
  D1 le, ln;
  losses<D1>(N, Vd.data(), K, T, fd.data(), E, edges, &le, &ln);
  const D1 L = w_eik * le + w_nc * ln;
  out[0] = L.v;
  out[1] = L.d[0];
}

// Marching Tetrahedra.  edges: the sorted unique edges (E pairs).  Writes up
// to vcap vertices (x, y, z) with their source edge index and up to tcap
// triangles; counts = (vertices, triangles) needed.  Returns 0, or -1 when a
// tet edge is missing from the edge list.
int orc_marching_tets(int64_t N, const double* V, int64_t K, const int32_t* T, const double* f,
                      int64_t E, const int32_t* edges, double* verts, int32_t* vert_edge,
                      int64_t vcap, int32_t* tris, int64_t tcap, int64_t* counts) {
  (void)N;
  // vertex id of each crossing edge, in edge order
  std::vector<int64_t> vid(E, -1);
  int64_t nv = 0;
  for (int64_t e = 0; e < E; ++e) {
    const int32_t a = edges[2 * e], b = edges[2 * e + 1];
    if ((f[a] > 0.0) == (f[b] > 0.0)) continue;
    vid[e] = nv;
    if (nv < vcap) {
      // zero of the linear interpolation along the edge
      for (int r = 0; r < 3; ++r)
        verts[3 * nv + r] = (V[3 * a + r] * f[b] - V[3 * b + r] * f[a]) / (f[b] - f[a]);
      if (vert_edge) vert_edge[nv] = (int32_t)e;
    }
    ++nv;
  }
  auto lookup = [&](int32_t x, int32_t y) -> int64_t {
    const std::pair<int32_t, int32_t> key(std::min(x, y), std::max(x, y));
    int64_t lo = 0, hi = E;
    while (lo < hi) {
      const int64_t mid = (lo + hi) / 2;
      const std::pair<int32_t, int32_t> m(edges[2 * mid], edges[2 * mid + 1]);
      if (m < key) lo = mid + 1; else hi = mid;
    }
    if (lo >= E || edges[2 * lo] != key.first || edges[2 * lo + 1] != key.second) return -1;
    return vid[lo];
  };
  auto det3 = [&](const int32_t o, const int32_t a, const int32_t b, const int32_t c) {
    double m[3][3];
    for (int r = 0; r < 3; ++r) {
      m[0][r] = V[3 * a + r] - V[3 * o + r];
      m[1][r] = V[3 * b + r] - V[3 * o + r];
      m[2][r] = V[3 * c + r] - V[3 * o + r];
    }
    return m[0][0] * (m[1][1] * m[2][2] - m[1][2] * m[2][1]) -
           m[0][1] * (m[1][0] * m[2][2] - m[1][2] * m[2][0]) +
           m[0][2] * (m[1][0] * m[2][1] - m[1][1] * m[2][0]);
  };
  int64_t nt = 0;
  auto emit = [&](int64_t x, int64_t y, int64_t z) {
    if (nt < tcap) {
      tris[3 * nt] = (int32_t)x;
      tris[3 * nt + 1] = (int32_t)y;
      tris[3 * nt + 2] = (int32_t)z;
    }
    ++nt;
  };
  for (int64_t k = 0; k < K; ++k) {
    const int32_t* t = T + 4 * k;
    bool pos[4];
    int np = 0;
    for (int i = 0; i < 4; ++i) {
      pos[i] = f[t[i]] > 0.0;
      np += pos[i] ? 1 : 0;
    }
    if (np == 0 || np == 4) continue;
    if (np == 1 || np == 3) {
      int o = -1, oth[3], m = 0;
      for (int i = 0; i < 4; ++i) {
        if (pos[i] == (np == 1)) o = i; else oth[m++] = i;
      }
      const int64_t x = lookup(t[o], t[oth[0]]), y = lookup(t[o], t[oth[1]]),
                    z = lookup(t[o], t[oth[2]]);
      if (x < 0 || y < 0 || z < 0) return -1;
      // (oa, ob, oc) faces away from o iff det(a - o, b - o, c - o) > 0; the
      // normal must point towards the positive side
      const double D = det3(t[o], t[oth[0]], t[oth[1]], t[oth[2]]);
      const bool flip = (np == 1) ? (D > 0.0) : (D < 0.0);
      if (flip) emit(x, z, y); else emit(x, y, z);
    } else {
      int P[2], Q[2], mp = 0, mq = 0;
      for (int i = 0; i < 4; ++i) {
        if (pos[i]) P[mp++] = i; else Q[mq++] = i;
      }
      const int p = P[0], q = P[1], r = Q[0], s_ = Q[1];
      const int64_t pr = lookup(t[p], t[r]), ps = lookup(t[p], t[s_]), qs = lookup(t[q], t[s_]),
                    qr = lookup(t[q], t[r]);
      if (pr < 0 || ps < 0 || qs < 0 || qr < 0) return -1;
      // (pr, ps, qs) and (pr, qs, qr) face the positive pair iff
      // det(q - p, r - p, s - p) < 0
      const double D = det3(t[p], t[q], t[r], t[s_]);
      if (D > 0.0) {
        emit(pr, qs, ps);
        emit(pr, qr, qs);
      } else {
        emit(pr, ps, qs);
        emit(pr, qs, qr);
      }
    }
  }
  counts[0] = nv;
  counts[1] = nt;
  return 0;
}

// Bounds of the vertices of the survivor tets (float min / max, exact):
// out = (xmin, ymin, zmin, xmax, ymax, zmax); (+inf, -inf) when empty.
void orc_survivor_bounds(const float* V, const int32_t* T, const int32_t* surv, int64_t nsurv,
                         float* out) {
  for (int r = 0; r < 3; ++r) {
    out[r] = INFINITY;
    out[3 + r] = -INFINITY;
  }
  for (int64_t i = 0; i < nsurv; ++i)
    for (int j = 0; j < 4; ++j) {
      const int64_t id = T[4 * (int64_t)surv[i] + j];
      for (int r = 0; r < 3; ++r) {
        out[r] = std::min(out[r], V[3 * id + r]);
        out[3 + r] = std::max(out[3 + r], V[3 * id + r]);
      }
    }
}

// The grid box [lo, hi] mapped per axis onto [b_lo, b_hi] = the bounds
// widened by pad * extent on each side (FP64); identity when the bounds are
// empty.
void orc_fit_grid(int64_t N, const float* V, const double* lo, const double* hi,
                  const float* aabb, double pad, double* out) {
  bool empty = false;
  for (int r = 0; r < 3; ++r) empty |= !(aabb[r] <= aabb[3 + r]);
  for (int64_t i = 0; i < N; ++i)
    for (int r = 0; r < 3; ++r) {
      const double x = V[3 * i + r];
      if (empty) {
        out[3 * i + r] = x;
        continue;
      }
      const double ext = (double)aabb[3 + r] - (double)aabb[r];
      const double blo = aabb[r] - pad * ext, bhi = aabb[3 + r] + pad * ext;
      out[3 * i + r] = blo + (x - lo[r]) * (bhi - blo) / (hi[r] - lo[r]);
    }
}

}  // extern "C"
